// The surrogate network on the tensor cores: a tcgen05 BF16 GEMM with TMA
// operand staging, an FP32 TMEM accumulator and fused epilogues (bias + GELU,
// GELU backward, split-K gradient accumulation, the final 256 -> 1 layer),
// plus the elementwise training kernels (minibatch gather, loss and head
// backward, bias gradients, Adam) and the C ABI of include/pd_surrogate.h.
#include "pd_internal.h"
#include "pd_surrogate.h"
#include "pd_tc.cuh"

#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

namespace pd {
namespace mlp {

using bf16 = __nv_bfloat16;

constexpr int kWidth = PD_MLP_WIDTH;
constexpr int kIn = PD_MLP_N_IN;
constexpr int kPad = PD_MLP_N_PAD;
constexpr int kInCols = PD_MLP_IN_COLS;      // network input row: 64 high parts, then 64 low parts
constexpr int kBM = 128, kBK = 64;
constexpr int kErrTimeout = 8;

// flat parameter offsets
constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + kWidth * kPad;
constexpr int OFF_W2 = OFF_B1 + kWidth;
constexpr int OFF_B2 = OFF_W2 + kWidth * kWidth;
constexpr int OFF_W3 = OFF_B2 + kWidth;
constexpr int OFF_B3 = OFF_W3 + kWidth * kWidth;
constexpr int OFF_W4 = OFF_B3 + kWidth;
constexpr int OFF_B4 = OFF_W4 + kWidth;
constexpr int N_PARAM = OFF_B4 + 1;
static_assert(N_PARAM == PD_MLP_N_PARAM, "parameter layout");

enum Epi { EPI_F32 = 0, EPI_F32_ATOMIC = 1, EPI_GELU = 2, EPI_GELU_BWD = 3, EPI_DOT = 4 };

struct GemmArgs {
    int M, N, K;                 // C[M x N] = A[M x K] . B[N x K]^T (rows of A from a_row0)
    int a_row0;
    int chunks_per_split;        // 64-wide K chunks per blockIdx.z
    int ldo;                     // row stride of out_f32 / out_bf16 / out_z / aux
    int ldt;                     // row stride of out_bf16_t ([N][ldt])
    const float* bias;
    const float* aux;            // EPI_GELU_BWD: pre-activation of this layer's input
    float* out_f32;
    bf16* out_bf16;
    bf16* out_bf16_t;
    float* out_z;
    const float* w_dot;          // EPI_DOT
    const float* b_dot;
    float* out_dot;
    int* err;
    unsigned long long wait_ns;
};

__host__ __device__ constexpr size_t gemm_smem_bytes(int BN, int S)
{
    return 1024 + (size_t)S * (kBM * kBK * 2 + (size_t)BN * kBK * 2) + (2 * S + 1) * 8 + 16 + kBM * 4;
}

// tanh(u) = 1 - 2 / (exp(2u) + 1) from the hardware base-2 exponential and
// reciprocal approximations: absolute error a few 1e-7 for every u (the ends go
// to +-1 through exp -> inf or 0), five instructions
__device__ __forceinline__ float tanh_acc(float u)
{
    float e, r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(u * 2.8853900817779268f));   // 2 / ln 2
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(e + 1.0f));
    return fmaf(-2.0f, r, 1.0f);
}

__device__ __forceinline__ float gelu_f(float x)
{
    const float u = 0.7978845608028654f * (x + 0.044715f * x * x * x);
    return 0.5f * x * (1.0f + tanh_acc(u));
}

__device__ __forceinline__ float gelu_grad_f(float x)
{
    const float u = 0.7978845608028654f * (x + 0.044715f * x * x * x);
    const float t = tanh_acc(u);
    return 0.5f * (1.0f + t) + 0.5f * x * (1.0f - t * t) * 0.7978845608028654f * (1.0f + 3.0f * 0.044715f * x * x);
}

// Hidden layers (their outputs are rounded to BF16) evaluate tanh with the
// hardware approximation tanh.approx.f32 (absolute error of order 2^-11, below
// the BF16 rounding step); the output layer keeps the accurate tanh_acc.
__device__ __forceinline__ float tanh_fast(float u)
{
    float t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(u));
    return t;
}

// Packed FP32 pairs (one instruction for two lanes of data on this part's
// FMA pipes) for the hidden-layer epilogue.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pk2(float a, float b) { f32x2 r; asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b)); return r; }
__device__ __forceinline__ void upk2(f32x2 v, float& a, float& b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v)); }
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) { f32x2 d; asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c)); return d; }
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) { f32x2 d; asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b)); return d; }
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) { f32x2 d; asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b)); return d; }

// gelu_fast of (x0 + b0, x1 + b1) as a pair: u = x (C + 0.044715 C x^2), tanh by
// tanh.approx per element, x (1/2 + t/2)
__device__ __forceinline__ void gelu_fast2(float& x0, float& x1, float b0, float b1)
{
    constexpr float kC = 0.7978845608028654f, kC3 = 0.044715f * 0.7978845608028654f;
    const f32x2 x = add2(pk2(x0, x1), pk2(b0, b1));
    const f32x2 u = mul2(x, fma2(mul2(x, x), pk2(kC3, kC3), pk2(kC, kC)));
    float u0, u1;
    upk2(u, u0, u1);
    const f32x2 h = fma2(pk2(tanh_fast(u0), tanh_fast(u1)), pk2(0.5f, 0.5f), pk2(0.5f, 0.5f));
    upk2(mul2(x, h), x0, x1);
}

__device__ __forceinline__ float gelu_fast(float x)
{
    const float u = 0.7978845608028654f * fmaf(0.044715f * x, x * x, x);
    return 0.5f * x * (1.0f + tanh_fast(u));
}

__device__ __forceinline__ float gelu_grad_fast(float x)
{
    const float u = 0.7978845608028654f * fmaf(0.044715f * x, x * x, x);
    const float t = tanh_fast(u);
    return 0.5f * (1.0f + t) + 0.5f * x * (1.0f - t * t) * 0.7978845608028654f * (1.0f + 3.0f * 0.044715f * x * x);
}

__device__ __forceinline__ void store_bf16x32(bf16* dst, const float (&h)[32])
{
    uint4* d = reinterpret_cast<uint4*>(dst);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        __nv_bfloat162 p0 = __floats2bfloat162_rn(h[8 * q + 0], h[8 * q + 1]);
        __nv_bfloat162 p1 = __floats2bfloat162_rn(h[8 * q + 2], h[8 * q + 3]);
        __nv_bfloat162 p2 = __floats2bfloat162_rn(h[8 * q + 4], h[8 * q + 5]);
        __nv_bfloat162 p3 = __floats2bfloat162_rn(h[8 * q + 6], h[8 * q + 7]);
        uint4 v;
        v.x = *reinterpret_cast<uint32_t*>(&p0);
        v.y = *reinterpret_cast<uint32_t*>(&p1);
        v.z = *reinterpret_cast<uint32_t*>(&p2);
        v.w = *reinterpret_cast<uint32_t*>(&p3);
        d[q] = v;
    }
}

__device__ __forceinline__ void store_bf16x16(bf16* dst, const float (&h)[16])
{
    uint4* d = reinterpret_cast<uint4*>(dst);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        __nv_bfloat162 p0 = __floats2bfloat162_rn(h[8 * q + 0], h[8 * q + 1]);
        __nv_bfloat162 p1 = __floats2bfloat162_rn(h[8 * q + 2], h[8 * q + 3]);
        __nv_bfloat162 p2 = __floats2bfloat162_rn(h[8 * q + 4], h[8 * q + 5]);
        __nv_bfloat162 p3 = __floats2bfloat162_rn(h[8 * q + 6], h[8 * q + 7]);
        uint4 v;
        v.x = *reinterpret_cast<uint32_t*>(&p0);
        v.y = *reinterpret_cast<uint32_t*>(&p1);
        v.z = *reinterpret_cast<uint32_t*>(&p2);
        v.w = *reinterpret_cast<uint32_t*>(&p3);
        d[q] = v;
    }
}

constexpr int kEpiWarps = 4;                  // one per TMEM lane quadrant
constexpr int kGemmThreads = 64 + 32 * kEpiWarps;

// One 128 x BN output tile per block: warp 0 stages A and B through an
// S-deep TMA ring, warp 1 owns the TMEM accumulator and issues the MMAs from
// one thread, warps 2..5 drain TMEM through the epilogue (lane quadrant =
// warp % 4).  With S = 2 two blocks fit on an SM, so one block's epilogue
// overlaps the other's loads and MMAs.  Every wait is bounded; a wait that
// runs out sets the error flag, lets the other roles finish and frees TMEM.
template <int BN, int EPI, int S>
__global__ void __launch_bounds__(kGemmThreads, (S <= 2 ? 2 : 1))
gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const GemmArgs a)
{
    constexpr int kStages = S;
    using namespace tc;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    constexpr uint32_t A_BYTES = kBM * kBK * 2, B_BYTES = BN * kBK * 2;
    uint8_t* sA = smem;
    uint8_t* sB = smem + kStages * A_BYTES;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sB + kStages * B_BYTES);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2 * kStages + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
    float* ydot_s = reinterpret_cast<float*>(tslot + 4);       // EPI_DOT: per-row partial sums [128]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
    const int n_chunks = (a.K + kBK - 1) / kBK;
    const int c_begin = blockIdx.z * a.chunks_per_split;
    const int nk = max(0, min(n_chunks, c_begin + a.chunks_per_split) - c_begin);
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + kStages), accf = smem_u32(bars + 2 * kStages);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(accf, 1);
        *abort_flag = 0;
        mbar_fence_init();
    }
    if (EPI == EPI_DOT && threadIdx.x < kBM) ydot_s[threadIdx.x] = 0.0f;
    if (warp == 1) tmem_alloc(smem_u32(tslot), BN);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == 0) {
        if (lane == 0 && nk > 0) {
            tma_prefetch_map(&tmA);
            tma_prefetch_map(&tmB);
            int issued = 0;
            for (int i = 0; i < nk; ++i) {
                const int s = i % kStages;
                if (i >= kStages && !mbar_wait(empty0 + 8 * s, ((i / kStages) & 1) ^ 1, a.wait_ns)) {
                    atomicOr(a.err, kErrTimeout);
                    *abort_flag = 1;
                    break;
                }
                if (*abort_flag) break;
                mbar_expect_tx(full0 + 8 * s, A_BYTES + B_BYTES);
                const int kx = (c_begin + i) * kBK;
                tma_load_2d(smem_u32(sA + s * A_BYTES), &tmA, full0 + 8 * s, kx, a.a_row0 + m0);
                tma_load_2d(smem_u32(sB + s * B_BYTES), &tmB, full0 + 8 * s, kx, n0);
                ++issued;
            }
            // the copies in flight land before the block can exit
            for (int i = max(0, issued - kStages); i < issued; ++i)
                if (!mbar_wait(full0 + 8 * (i % kStages), (i / kStages) & 1, a.wait_ns)) atomicOr(a.err, kErrTimeout);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16_f32(kBM, BN);
            for (int i = 0; i < nk; ++i) {
                const int s = i % kStages;
                if (!mbar_wait(full0 + 8 * s, (i / kStages) & 1, a.wait_ns)) {
                    atomicOr(a.err, kErrTimeout);
                    *abort_flag = 1;
                    break;
                }
                tc_fence_after();
                const uint64_t ad = sdesc_sw128(smem_u32(sA + s * A_BYTES));
                const uint64_t bd = sdesc_sw128(smem_u32(sB + s * B_BYTES));
#pragma unroll
                for (int kk = 0; kk < kBK / 16; ++kk)
                    mma_bf16(tmem, ad + 2 * kk, bd + 2 * kk, idesc, (i > 0 || kk > 0) ? 1u : 0u);
                mma_commit(empty0 + 8 * s);
            }
            mma_commit(accf);
        }
    } else {
        const int quad = warp & 3;
        const int half = (warp - 2) >> 2;            // 0: one warp per quadrant covers every column
        const int rl = quad * 32 + lane;
        const int row = m0 + rl;
        int ok = 1;
        if (lane == 0) {
            ok = mbar_wait(accf, 0, a.wait_ns) ? 1 : 0;
            if (!ok) atomicOr(a.err, kErrTimeout);
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        tc_fence_after();
        const bool live = ok && !*abort_flag;
        const bool in = live && row < a.M;
        const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16);
        constexpr int CW = BN / (kEpiWarps / 4);    // columns of this warp
        float ydot = 0.0f;
        if (live) {
#pragma unroll 1
            for (int c = 0; c < CW / 16; ++c) {
                const int col = half * CW + c * 16;
                float v[16];
                tmem_ld16(tbase + col, v);
                if (!in) continue;
                const int nb = n0 + col;
                if (EPI == EPI_F32) {
                    float* o = a.out_f32 + (size_t)row * a.ldo + nb;
#pragma unroll
                    for (int k = 0; k < 16; k += 4) {
                        float4 q = make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
                        if (a.bias) { q.x += a.bias[nb + k]; q.y += a.bias[nb + k + 1]; q.z += a.bias[nb + k + 2]; q.w += a.bias[nb + k + 3]; }
                        *reinterpret_cast<float4*>(o + k) = q;
                    }
                } else if (EPI == EPI_F32_ATOMIC) {
                    float* o = a.out_f32 + (size_t)row * a.ldo + nb;
#pragma unroll
                    for (int k = 0; k < 16; ++k) atomicAdd(o + k, v[k]);
                } else if (EPI == EPI_GELU) {
#pragma unroll
                    for (int k = 0; k < 16; ++k) v[k] += a.bias[nb + k];
                    if (a.out_z) {
                        float* o = a.out_z + (size_t)row * a.ldo + nb;
#pragma unroll
                        for (int k = 0; k < 16; k += 4) *reinterpret_cast<float4*>(o + k) = make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
                    }
#pragma unroll
                    for (int k = 0; k < 16; ++k) v[k] = gelu_fast(v[k]);
                    if (a.out_bf16) store_bf16x16(a.out_bf16 + (size_t)row * a.ldo + nb, v);
                    if (a.out_bf16_t) {
#pragma unroll
                        for (int k = 0; k < 16; ++k) a.out_bf16_t[(size_t)(nb + k) * a.ldt + row] = __float2bfloat16_rn(v[k]);
                    }
                } else if (EPI == EPI_GELU_BWD) {
                    const float* z = a.aux + (size_t)row * a.ldo + nb;
#pragma unroll
                    for (int k = 0; k < 16; k += 4) {
                        const float4 q = *reinterpret_cast<const float4*>(z + k);
                        v[k] *= gelu_grad_fast(q.x);
                        v[k + 1] *= gelu_grad_fast(q.y);
                        v[k + 2] *= gelu_grad_fast(q.z);
                        v[k + 3] *= gelu_grad_fast(q.w);
                    }
                    store_bf16x16(a.out_bf16 + (size_t)row * a.ldo + nb, v);
#pragma unroll
                    for (int k = 0; k < 16; ++k) a.out_bf16_t[(size_t)(nb + k) * a.ldt + row] = __float2bfloat16_rn(v[k]);
                } else {   // EPI_DOT
#pragma unroll
                    for (int k = 0; k < 16; ++k) ydot = fmaf(gelu_f(v[k] + a.bias[nb + k]), a.w_dot[nb + k], ydot);
                }
            }
            // column groups of a row meet in shared memory (one group: a plain store)
            if (EPI == EPI_DOT && in) atomicAdd(&ydot_s[rl], ydot);
        }
        if (EPI == EPI_DOT) {
            asm volatile("bar.sync 1, %0;" ::"r"(32 * kEpiWarps) : "memory");
            if (half == 0 && in) a.out_dot[row] = ydot_s[rl] + *a.b_dot;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, BN);
    }
}

// ---------------------------------------------------------------------------
// elementwise training kernels

// Minibatch rows r of [B][128] from sample (a (s0 + r) + b) mod n (or row r of
// X when a == 0), the transposed high parts [64][ld] and the targets; rows at
// or past n_valid are zero.  Block: 64 rows, 256 threads.
__global__ void __launch_bounds__(256) gather_kernel(const bf16* __restrict__ X, const float* __restrict__ T,
                                                     long long n, unsigned long long ma, unsigned long long mb,
                                                     long long s0, int n_valid, int ld,
                                                     bf16* __restrict__ Xb, bf16* __restrict__ Xbt, float* __restrict__ tb)
{
    __shared__ bf16 tile[64][kPad + 2];
    const int r0 = blockIdx.x * 64;
    for (int e = threadIdx.x; e < 64 * 16; e += blockDim.x) {
        const int r = e >> 4, q = e & 15;
        const int row = r0 + r;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (row < n_valid) {
            long long src = ma ? (long long)((ma * (unsigned long long)(s0 + row) + mb) % (unsigned long long)n) : (long long)row;
            v = reinterpret_cast<const uint4*>(X + (size_t)src * kInCols)[q];
            if (q == 0 && T) tb[row] = T[src];
        } else if (q == 0) {
            tb[row] = 0.0f;
        }
        reinterpret_cast<uint4*>(Xb + (size_t)row * kInCols)[q] = v;
        if (q < 8) {
            const bf16* h = reinterpret_cast<const bf16*>(&v);
#pragma unroll
            for (int k = 0; k < 8; ++k) tile[r][q * 8 + k] = h[k];
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 64 * 64; e += blockDim.x) {
        const int c = e >> 6, r = e & 63;
        Xbt[(size_t)c * ld + r0 + r] = tile[r][c];
    }
}

// Output layer and loss for 32 rows per block (8 warps, 4 rows each):
// y = w4 . g(z3) + b4, d = 2 (y - t)/n, dZ3 = d w4 g'(z3) (row-major and
// transposed BF16 with row stride ld), gradients of w4, b4, and the summed
// squared error.
__global__ void __launch_bounds__(256) head_kernel(const float* __restrict__ Z3, const float* __restrict__ tb,
                                                   const float* __restrict__ w4, const float* __restrict__ theta,
                                                   int n_valid, int ld, float inv_n,
                                                   bf16* __restrict__ dZ3, bf16* __restrict__ dZ3t,
                                                   float* __restrict__ grad, float* __restrict__ loss_acc)
{
    __shared__ bf16 tile[32][kWidth + 8];
    __shared__ float gw4[kWidth];
    __shared__ float red[2];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = threadIdx.x; k < kWidth; k += blockDim.x) gw4[k] = 0.0f;
    if (threadIdx.x < 2) red[threadIdx.x] = 0.0f;
    __syncthreads();
    const float b4 = theta[OFF_B4];
    float gw[8] = { 0, 0, 0, 0, 0, 0, 0, 0 };
    float gb = 0.0f, sq = 0.0f;
    for (int rr = 0; rr < 4; ++rr) {
        const int rl = warp * 4 + rr;
        const int row = blockIdx.x * 32 + rl;
        const float* z = Z3 + (size_t)row * kWidth + lane * 8;
        float zv[8], h[8];
        const float4 q0 = reinterpret_cast<const float4*>(z)[0], q1 = reinterpret_cast<const float4*>(z)[1];
        zv[0] = q0.x; zv[1] = q0.y; zv[2] = q0.z; zv[3] = q0.w; zv[4] = q1.x; zv[5] = q1.y; zv[6] = q1.z; zv[7] = q1.w;
        float part = 0.0f;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            h[k] = gelu_f(zv[k]);
            part = fmaf(h[k], w4[lane * 8 + k], part);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        const bool valid = row < n_valid;
        const float e = valid ? (part + b4 - tb[row]) : 0.0f;
        const float d = 2.0f * e * inv_n;
        sq += e * e;
        gb += d;
        float g[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            g[k] = d * w4[lane * 8 + k] * gelu_grad_f(zv[k]);
            gw[k] = fmaf(d, h[k], gw[k]);
        }
        __nv_bfloat162* dst = reinterpret_cast<__nv_bfloat162*>(dZ3 + (size_t)row * kWidth + lane * 8);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            __nv_bfloat162 pk = __floats2bfloat162_rn(g[2 * k], g[2 * k + 1]);
            dst[k] = pk;
            tile[rl][lane * 8 + 2 * k] = pk.x;
            tile[rl][lane * 8 + 2 * k + 1] = pk.y;
        }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) atomicAdd(&gw4[lane * 8 + k], gw[k]);
    if (lane == 0) {
        atomicAdd(&red[0], gb);
        atomicAdd(&red[1], sq);
    }
    __syncthreads();
    // transposed copy: column c of the tile is 32 consecutive rows of dZ3t
    for (int e = threadIdx.x; e < kWidth * 32; e += blockDim.x) {
        const int c = e >> 5, r = e & 31;
        dZ3t[(size_t)c * ld + blockIdx.x * 32 + r] = tile[r][c];
    }
    for (int k = threadIdx.x; k < kWidth; k += blockDim.x) atomicAdd(&grad[OFF_W4 + k], gw4[k]);
    if (threadIdx.x == 0) {
        atomicAdd(&grad[OFF_B4], red[0]);
        atomicAdd(loss_acc, red[1]);
    }
}

// Bias gradients: db[n] = sum over the minibatch of dZ^T[n][:], one block per
// (unit, layer).
__global__ void __launch_bounds__(256) bias_grad_kernel(const bf16* __restrict__ t1, const bf16* __restrict__ t2,
                                                        const bf16* __restrict__ t3, int B, int ld, float* __restrict__ grad)
{
    const int n = blockIdx.x, layer = blockIdx.y;
    const bf16* src = (layer == 0 ? t1 : layer == 1 ? t2 : t3) + (size_t)n * ld;
    float s = 0.0f;
    for (int b = threadIdx.x; b < B; b += blockDim.x) s += __bfloat162float(src[b]);
    __shared__ float red[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        const int off = layer == 0 ? OFF_B1 : layer == 1 ? OFF_B2 : OFF_B3;
        grad[off + n] = t;
    }
}

// Adam on every parameter (the gradient is consumed and zeroed), then the
// BF16 operand copies: W1, W2, W3 row-major, W2^T and W3^T, and w4 rounded
// to BF16 (held as FP32).
__global__ void adam_kernel(float* __restrict__ theta, float* __restrict__ grad, float* __restrict__ m1,
                            float* __restrict__ m2, const float* __restrict__ lr_ptr, float lr_host, float c1, float c2,
                            int do_update, bf16* __restrict__ W1b, bf16* __restrict__ W2b, bf16* __restrict__ W3b,
                            bf16* __restrict__ W2t, bf16* __restrict__ W3t, float* __restrict__ w4b)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N_PARAM) return;
    float th = theta[i];
    if (do_update) {
        const float lr = lr_ptr ? *lr_ptr : lr_host;
        const float g = grad[i];
        const float a = 0.9f * m1[i] + 0.1f * g;
        const float b = 0.999f * m2[i] + 0.001f * g * g;
        m1[i] = a;
        m2[i] = b;
        th -= lr * (a * c1) / (sqrtf(b * c2) + 1e-8f);
        theta[i] = th;
        grad[i] = 0.0f;
    }
    const bf16 h = __float2bfloat16_rn(th);
    if (i < OFF_B1) {
        // the high and the low input parts meet the same first-layer weights
        const int n = i / kPad, k = i - n * kPad;
        W1b[n * kInCols + k] = h;
        W1b[n * kInCols + kPad + k] = h;
    } else if (i >= OFF_W2 && i < OFF_B2) {
        const int k = i - OFF_W2;
        W2b[k] = h;
        W2t[(k % kWidth) * kWidth + k / kWidth] = h;
    } else if (i >= OFF_W3 && i < OFF_B3) {
        const int k = i - OFF_W3;
        W3b[k] = h;
        W3t[(k % kWidth) * kWidth + k / kWidth] = h;
    } else if (i >= OFF_W4 && i < OFF_B4) {
        w4b[i - OFF_W4] = __bfloat162float(h);
    }
}

// Feature statistics: per-feature sum and sum of squares (FP64) and sum |y|.
__global__ void norm_stats_kernel(const float* __restrict__ X, const float* __restrict__ y, long long n,
                                  double* __restrict__ acc)
{
    __shared__ double s1[kIn + 1], s2[kIn];
    for (int k = threadIdx.x; k < kIn + 1; k += blockDim.x) s1[k] = 0.0;
    for (int k = threadIdx.x; k < kIn; k += blockDim.x) s2[k] = 0.0;
    __syncthreads();
    double a1[kIn], a2[kIn], ay = 0.0;
    for (int k = 0; k < kIn; ++k) { a1[k] = 0.0; a2[k] = 0.0; }
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
        const float* x = X + r * kIn;
        for (int k = 0; k < kIn; ++k) {
            const double v = x[k];
            a1[k] += v;
            a2[k] += v * v;
        }
        ay += fabs((double)y[r]);
    }
    for (int k = 0; k < kIn; ++k) {
        atomicAdd(&s1[k], a1[k]);
        atomicAdd(&s2[k], a2[k]);
    }
    atomicAdd(&s1[kIn], ay);
    __syncthreads();
    for (int k = threadIdx.x; k < kIn; k += blockDim.x) {
        atomicAdd(&acc[k], s1[k]);
        atomicAdd(&acc[kIn + 1 + k], s2[k]);
    }
    if (threadIdx.x == 0) atomicAdd(&acc[kIn], s1[kIn]);
}

// v = (x - mu)/sigma in FP32 into the network input row [128]: hi = bf16(v)
// at column k, lo = bf16(v - hi) at column 64 + k (padding zero); y/y_scale.
__global__ void pack_kernel(const float* __restrict__ X, const float* __restrict__ y, long long n,
                            const float* __restrict__ norm, bf16* __restrict__ Xo, float* __restrict__ to)
{
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= n * kPad) return;
    const long long r = e / kPad;
    const int k = (int)(e - r * kPad);
    float v = 0.0f;
    if (k < kIn) v = (X[r * kIn + k] - norm[k]) / norm[kIn + k];
    const bf16 hi = __float2bfloat16_rn(v);
    Xo[r * kInCols + k] = hi;
    Xo[r * kInCols + kPad + k] = __float2bfloat16_rn(v - __bfloat162float(hi));
    if (k == 0 && y && to) to[r] = y[r] / norm[2 * kIn];
}

// Fan-in uniform initialisation: every weight and bias of a layer with fan-in
// f is drawn from U(-1/sqrt f, 1/sqrt f) (f = 35 for the first layer, 256
// after it); the padding columns of W1 stay zero.  The draw for parameter i is
// splitmix64(seed + (i + 1) * golden) scaled to [0, 1).
__global__ void init_kernel(float* __restrict__ theta, unsigned long long seed)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N_PARAM) return;
    unsigned long long z = seed + (unsigned long long)(i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
    double bound;
    if (i < OFF_B1) bound = (i % kPad) < kIn ? 1.0 / sqrt((double)kIn) : 0.0;
    else if (i < OFF_W2) bound = 1.0 / sqrt((double)kIn);
    else bound = 1.0 / sqrt((double)kWidth);
    theta[i] = (float)((2.0 * u - 1.0) * bound);
}

// learning rate of step s (device-side, so a captured step graph reads it)
__global__ void lr_kernel(float* lr, long long s, long long total, float lr_max)
{
    const long long warm = std::max<long long>(1, total / 20);
    float v;
    if (s < warm) v = lr_max * (float)(s + 1) / (float)warm;
    else v = 0.5f * lr_max * (1.0f + cosf(3.14159265358979f * (float)(s - warm) / (float)std::max<long long>(1, total - warm)));
    *lr = v;
}

// ---------------------------------------------------------------------------
// Fused network forward: one persistent block per SM loops over 128-row tiles
// and runs all three layers on chip.  The 64 KB activation buffer holds the
// tile's input (TMA) and then each hidden layer's BF16 output, written by the
// epilogue warps in the same 128-byte-swizzled K-major layout the TMA uses
// (16-byte unit j of row r at unit j ^ (r & 7)), so it is the next MMA's A
// operand directly.  Weight chunks [256 x 64] stream through a TMA ring.

struct FusedArgs {
    long long n;
    int n_tiles;
    const float* b1;
    const float* b2;
    const float* b3;
    const float* w4;
    const float* b4;
    float* y;
    int* err;
    unsigned long long wait_ns;
};

constexpr int kFS = 3;                         // weight ring stages
constexpr int kFEpi = 8;                       // epilogue warps: two per TMEM lane quadrant
constexpr int kFThreads = 64 + 32 * kFEpi;
constexpr uint32_t kActChunk = 128 * 64 * 2;   // [128 rows][64] BF16
constexpr uint32_t kActBytes = 4 * kActChunk;  // one tile's activations
constexpr uint32_t kWChunk = 256 * 64 * 2;     // [256 rows][64] BF16
constexpr int kFBars = 2 * kFS + 12;

__host__ __device__ constexpr size_t fused_smem_bytes()
{
    return 1024 + 2 * (size_t)kActBytes + (size_t)kFS * kWChunk + kFBars * 8 + 16 + 2 * 128 * 4;
}
static_assert(fused_smem_bytes() <= 232448, "fused MLP shared memory");

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void fence_async_shared()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Hidden-layer epilogue of 32 accumulator columns [col0, col0 + 32) of row r:
// bias, GELU, BF16, stored into the next layer's operand in the
// 128-byte-swizzled K-major layout (16-byte unit j of row r at j ^ (r & 7)).
__device__ __forceinline__ void epi_hidden32(const uint32_t (&u)[32], int col0, const float* bias, uint8_t* act, int r)
{
    float v[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) v[k] = __uint_as_float(u[k]);
    const float4* bq = reinterpret_cast<const float4*>(bias + col0);
#pragma unroll
    for (int k4 = 0; k4 < 8; ++k4) {
        const float4 bb = __ldg(bq + k4);
        gelu_fast2(v[4 * k4 + 0], v[4 * k4 + 1], bb.x, bb.y);
        gelu_fast2(v[4 * k4 + 2], v[4 * k4 + 3], bb.z, bb.w);
    }
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        uint4 q;
        __nv_bfloat162 p0 = __floats2bfloat162_rn(v[8 * h + 0], v[8 * h + 1]);
        __nv_bfloat162 p1 = __floats2bfloat162_rn(v[8 * h + 2], v[8 * h + 3]);
        __nv_bfloat162 p2 = __floats2bfloat162_rn(v[8 * h + 4], v[8 * h + 5]);
        __nv_bfloat162 p3 = __floats2bfloat162_rn(v[8 * h + 6], v[8 * h + 7]);
        q.x = *reinterpret_cast<uint32_t*>(&p0);
        q.y = *reinterpret_cast<uint32_t*>(&p1);
        q.z = *reinterpret_cast<uint32_t*>(&p2);
        q.w = *reinterpret_cast<uint32_t*>(&p3);
        const int col = col0 + 8 * h;
        const int kc = col >> 6, j = (col & 63) >> 3;
        *reinterpret_cast<uint4*>(act + kc * kActChunk + r * 128 + ((j ^ (r & 7)) << 4)) = q;
    }
}

// GELU of a pair with the accurate tanh of tanh_acc (exp2 and reciprocal per
// element, the rest on packed FP32 pairs): x (1/2 + t/2), t = 1 - 2 / (exp(2u) + 1),
// u = C x (1 + 0.044715 x^2)
__device__ __forceinline__ f32x2 gelu_acc2(f32x2 x)
{
    constexpr float kU2 = 0.7978845608028654f * 2.8853900817779268f;   // C * 2 / ln 2
    constexpr float kU23 = 0.044715f * kU2;
    const f32x2 z = mul2(x, fma2(mul2(x, x), pk2(kU23, kU23), pk2(kU2, kU2)));
    float z0, z1, e0, e1;
    upk2(z, z0, z1);
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e0) : "f"(z0));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e1) : "f"(z1));
    float d0, d1, r0, r1;
    upk2(add2(pk2(e0, e1), pk2(1.0f, 1.0f)), d0, d1);
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(d0));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r1) : "f"(d1));
    const f32x2 t = fma2(pk2(r0, r1), pk2(-2.0f, -2.0f), pk2(1.0f, 1.0f));
    return mul2(x, fma2(t, pk2(0.5f, 0.5f), pk2(0.5f, 0.5f)));
}

// Output-layer epilogue: part + sum over 32 columns of w4 * GELU(acc + b3), the
// even and odd columns accumulated as one packed pair
__device__ __forceinline__ float epi_dot32(const uint32_t (&u)[32], int col0, const float* b3, const float* w4, float part)
{
    const float4* bq = reinterpret_cast<const float4*>(b3 + col0);
    const float4* wq = reinterpret_cast<const float4*>(w4 + col0);
    f32x2 acc = pk2(part, 0.0f);
#pragma unroll
    for (int k4 = 0; k4 < 8; ++k4) {
        const float4 bb = __ldg(bq + k4), ww = __ldg(wq + k4);
        const f32x2 x01 = add2(pk2(__uint_as_float(u[4 * k4 + 0]), __uint_as_float(u[4 * k4 + 1])), pk2(bb.x, bb.y));
        const f32x2 x23 = add2(pk2(__uint_as_float(u[4 * k4 + 2]), __uint_as_float(u[4 * k4 + 3])), pk2(bb.z, bb.w));
        acc = fma2(gelu_acc2(x01), pk2(ww.x, ww.y), acc);
        acc = fma2(gelu_acc2(x23), pk2(ww.z, ww.w), acc);
    }
    float a0, a1;
    upk2(acc, a0, a1);
    return a0 + a1;
}

// Two tiles in flight per block (slots 0 and 1, each with its own activation
// buffer and 256-column TMEM accumulator), processed layer by layer in the
// job order (A, L1), (B, L1), (A, L2), (B, L2), (A, L3), (B, L3) for each pair
// of tiles A = blockIdx.x + 2 p gridDim.x, B = A + gridDim.x: while the
// epilogue warps turn one slot's accumulator into the next layer's operand,
// the tensor core runs the other slot's layer.  Every role walks the same job
// order; per slot, barrier phases count tiles (input, activation free) or
// jobs (accumulator full, epilogue done).
__global__ void __launch_bounds__(kFThreads, 1)
mlp_fused_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmW1,
                 const __grid_constant__ CUtensorMap tmW2, const __grid_constant__ CUtensorMap tmW3, const FusedArgs a)
{
    using namespace tc;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* act0 = smem;                                   // slot s at act0 + s kActBytes
    uint8_t* ring = smem + 2 * kActBytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(ring + kFS * kWChunk);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + kFBars);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
    float* ydot0 = reinterpret_cast<float*>(tslot + 4);    // [2][128]: second-half partial sums

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t b0 = smem_u32(bars);
    auto wfull = [&](int s) { return b0 + 8 * s; };
    auto wempty = [&](int s) { return b0 + 8 * (kFS + s); };
    const uint32_t bslot = b0 + 8 * (2 * kFS);              // six per-slot barriers, two slots each
    auto xfull = [&](int s) { return bslot + 8 * (0 + s); };
    auto accfull = [&](int s) { return bslot + 8 * (2 + s); };
    auto epidone = [&](int s) { return bslot + 8 * (4 + s); };
    auto actfree = [&](int s) { return bslot + 8 * (6 + s); };
    auto ydotready = [&](int s) { return bslot + 8 * (8 + s); };
    const uint32_t done = bslot + 8 * 10;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kFS; ++s) {
            mbar_init(wfull(s), 1);
            mbar_init(wempty(s), 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(xfull(s), 1);
            mbar_init(accfull(s), 1);
            mbar_init(epidone(s), kFEpi);
            mbar_init(actfree(s), 1);
            mbar_init(ydotready(s), kFEpi / 2);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        mbar_fence_init();
    }
    if (warp == 1) tmem_alloc(smem_u32(tslot), 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    // a wait that gives up (or sees another role give up) ends this role's loop
    auto wait = [&](uint32_t bar, uint32_t parity) -> bool {
        if (*abort_flag) return false;
        if (mbar_wait(bar, parity, a.wait_ns)) return true;
        atomicOr(a.err, kErrTimeout);
        *abort_flag = 1;
        return false;
    };
    const int n_pairs = (a.n_tiles - (int)blockIdx.x + 2 * (int)gridDim.x - 1) / (2 * (int)gridDim.x);
    auto tile_of = [&](int pi, int s) { return (int)blockIdx.x + (2 * pi + s) * (int)gridDim.x; };

    if (warp == 0) {
        if (lane == 0) {
            tma_prefetch_map(&tmX);
            tma_prefetch_map(&tmW1);
            tma_prefetch_map(&tmW2);
            tma_prefetch_map(&tmW3);
            int wc = 0;
            int last_x[2] = { -1, -1 };          // pair of the last input copy issued per slot
            bool ok = true;
            for (int pi = 0; ok && pi < n_pairs; ++pi) {
                for (int s = 0; ok && s < 2; ++s) {
                    const int tile = tile_of(pi, s);
                    if (tile >= a.n_tiles) continue;
                    if (pi > 0 && !(ok = wait(actfree(s), (pi - 1) & 1))) break;
                    uint8_t* act = act0 + s * kActBytes;
                    mbar_expect_tx(xfull(s), 2 * kActChunk);
                    tma_load_2d(smem_u32(act), &tmX, xfull(s), 0, tile * 128);
                    tma_load_2d(smem_u32(act + kActChunk), &tmX, xfull(s), 64, tile * 128);
                    last_x[s] = pi;
                }
                for (int L = 0; ok && L < 3; ++L) {
                    const CUtensorMap* mp = L == 0 ? &tmW1 : (L == 1 ? &tmW2 : &tmW3);
                    const int nk = L == 0 ? 2 : 4;
                    for (int s = 0; ok && s < 2; ++s) {
                        if (tile_of(pi, s) >= a.n_tiles) continue;
                        for (int kc = 0; kc < nk; ++kc, ++wc) {
                            const int st = wc % kFS;
                            if (wc >= kFS && !(ok = wait(wempty(st), ((wc / kFS) & 1) ^ 1))) break;
                            mbar_expect_tx(wfull(st), kWChunk);
                            tma_load_2d(smem_u32(ring + st * kWChunk), mp, wfull(st), kc * 64, 0);
                        }
                    }
                }
            }
            // the copies in flight land before the block can exit
            for (int k = max(0, wc - kFS); k < wc; ++k)
                if (!mbar_wait(wfull(k % kFS), (k / kFS) & 1, a.wait_ns)) atomicOr(a.err, kErrTimeout);
            for (int s = 0; s < 2; ++s)
                if (last_x[s] >= 0 && !mbar_wait(xfull(s), last_x[s] & 1, a.wait_ns)) atomicOr(a.err, kErrTimeout);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16_f32(128, 256);
            int wc = 0;
            bool ok = true, issued = false;
            for (int pi = 0; ok && pi < n_pairs; ++pi) {
                for (int L = 0; ok && L < 3; ++L) {
                    for (int s = 0; ok && s < 2; ++s) {
                        if (tile_of(pi, s) >= a.n_tiles) continue;
                        const int job = 3 * pi + L;              // jobs of this slot so far
                        if (L == 0) {
                            // the slot's accumulator is free once the epilogue finished the previous tile
                            if (pi > 0 && !(ok = wait(epidone(s), (job - 1) & 1))) break;
                            if (!(ok = wait(xfull(s), pi & 1))) break;
                        } else {
                            if (!(ok = wait(epidone(s), (job - 1) & 1))) break;
                        }
                        tc_fence_after();
                        const uint8_t* act = act0 + s * kActBytes;
                        const uint32_t acc = tmem + (uint32_t)(s * 256);
                        const int nk = L == 0 ? 2 : 4;
                        for (int kc = 0; kc < nk; ++kc, ++wc) {
                            const int st = wc % kFS;
                            if (!(ok = wait(wfull(st), (wc / kFS) & 1))) break;
                            tc_fence_after();
                            const uint64_t ad = sdesc_sw128(smem_u32(act + kc * kActChunk));
                            const uint64_t bd = sdesc_sw128(smem_u32(ring + st * kWChunk));
#pragma unroll
                            for (int kk = 0; kk < kBK / 16; ++kk)
                                mma_bf16(acc, ad + 2 * kk, bd + 2 * kk, idesc, (kc > 0 || kk > 0) ? 1u : 0u);
                            mma_commit(wempty(st));
                            issued = true;
                        }
                        if (!ok) break;
                        mma_commit(accfull(s));
                        if (L == 2) mma_commit(actfree(s));
                    }
                }
            }
            // every MMA issued has completed before TMEM is freed
            if (issued) {
                mma_commit(done);
                if (!mbar_wait(done, 0, a.wait_ns)) atomicOr(a.err, kErrTimeout);
            }
        }
    } else {
        const int quad = warp & 3;
        const int half = (warp - 2) >> 2;
        const int r = quad * 32 + lane;
        bool ok = true;
        for (int pi = 0; ok && pi < n_pairs; ++pi) {
            for (int L = 0; ok && L < 3; ++L) {
                for (int s = 0; ok && s < 2; ++s) {
                    const int tile = tile_of(pi, s);
                    if (tile >= a.n_tiles) continue;
                    const int job = 3 * pi + L;
                    int w_ok = 1;
                    if (lane == 0) w_ok = wait(accfull(s), job & 1) ? 1 : 0;
                    w_ok = __shfl_sync(0xffffffffu, w_ok, 0);
                    if (!w_ok) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t tbase = tmem + (uint32_t)(s * 256) + ((uint32_t)(quad * 32) << 16);
                    uint8_t* act = act0 + s * kActBytes;
                    float* ydot = ydot0 + s * 128;
                    // the warp's 128 columns in four 32-column TMEM loads, each
                    // issued while the previous piece is processed
                    const int colw = half * 128;
                    uint32_t ra[32], rb[32];
                    tmem_ld32_issue(tbase + colw, ra);
                    tmem_ld_wait();
                    tmem_reg_fence(ra);
                    if (L < 2) {
                        const float* bias = L == 0 ? a.b1 : a.b2;
                        tmem_ld32_issue(tbase + colw + 32, rb);
                        epi_hidden32(ra, colw, bias, act, r);
                        tmem_ld_wait();
                        tmem_reg_fence(rb);
                        tmem_ld32_issue(tbase + colw + 64, ra);
                        epi_hidden32(rb, colw + 32, bias, act, r);
                        tmem_ld_wait();
                        tmem_reg_fence(ra);
                        tmem_ld32_issue(tbase + colw + 96, rb);
                        epi_hidden32(ra, colw + 64, bias, act, r);
                        tmem_ld_wait();
                        tmem_reg_fence(rb);
                        epi_hidden32(rb, colw + 96, bias, act, r);
                        fence_async_shared();
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(epidone(s));
                    } else {
                        float part = 0.0f;
                        tmem_ld32_issue(tbase + colw + 32, rb);
                        part = epi_dot32(ra, colw, a.b3, a.w4, part);
                        tmem_ld_wait();
                        tmem_reg_fence(rb);
                        tmem_ld32_issue(tbase + colw + 64, ra);
                        part = epi_dot32(rb, colw + 32, a.b3, a.w4, part);
                        tmem_ld_wait();
                        tmem_reg_fence(ra);
                        tmem_ld32_issue(tbase + colw + 96, rb);
                        part = epi_dot32(ra, colw + 64, a.b3, a.w4, part);
                        tmem_ld_wait();
                        tmem_reg_fence(rb);
                        part = epi_dot32(rb, colw + 96, a.b3, a.w4, part);
                        tc_fence_before();
                        if (half == 1) {
                            // the second column half hands its partial sums over (bounded wait on the other side)
                            ydot[r] = part;
                            __syncwarp();
                            if (lane == 0) {
                                mbar_arrive(epidone(s));
                                mbar_arrive(ydotready(s));
                            }
                        } else {
                            __syncwarp();
                            if (lane == 0) mbar_arrive(epidone(s));
                            int y_ok = 1;
                            if (lane == 0) y_ok = wait(ydotready(s), pi & 1) ? 1 : 0;
                            y_ok = __shfl_sync(0xffffffffu, y_ok, 0);
                            if (!y_ok) { ok = false; break; }
                            const long long row = (long long)tile * 128 + r;
                            if (row < a.n) a.y[row] = part + ydot[r] + *a.b4;
                        }
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

// S = 2 for the short products (K <= 256: every forward and input-gradient
// GEMM), S = 4 for the weight gradients whose K is the minibatch
template <int BN, int EPI, int S = 2>
cudaError_t launch_gemm(const CUtensorMap& ta, const CUtensorMap& tb, const GemmArgs& a, int splits, cudaStream_t st)
{
    static bool attr = false;
    const size_t smem = gemm_smem_bytes(BN, S);
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(gemm_kernel<BN, EPI, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 grid((a.M + kBM - 1) / kBM, a.N / BN, splits);
    gemm_kernel<BN, EPI, S><<<grid, kGemmThreads, smem, st>>>(ta, tb, a);
    return cudaGetLastError();
}

}  // namespace mlp
}  // namespace pd

// ---------------------------------------------------------------------------
// host object

using namespace pd::mlp;

namespace {

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

cudaError_t get_encoder()
{
    if (g_encode) return cudaSuccess;
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorSymbolNotFound;
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    return cudaSuccess;
}

// K-major BF16 operand [rows][ld] read in [box_rows][64] tiles with 128-byte
// swizzling; rows past `rows` and columns past `cols` read as zero.
bool make_map(CUtensorMap* m, const void* ptr, long long rows, int cols, int ld, int box_rows)
{
    if (!g_encode || ((uintptr_t)ptr & 15) || (ld * 2) % 16 || box_rows > 256 || rows < 1) return false;
    cuuint64_t dims[2] = { (cuuint64_t)cols, (cuuint64_t)rows };
    cuuint64_t strides[1] = { (cuuint64_t)ld * 2 };
    cuuint32_t box[2] = { 64, (cuuint32_t)box_rows };
    cuuint32_t es[2] = { 1, 1 };
    CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

struct Maps {
    CUtensorMap Xb, W1, H1, W2, H2, W3, dZ3t, H2t, dZ3, W3t, dZ2t, H1t, dZ2, W2t, dZ1t, Xbt, I1, I2;
};

}  // namespace

struct pd_mlp {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string last;
    int cap = 0;                     // max minibatch rows
    int chunk = 65536;               // inference rows per pass
    float *theta = nullptr, *grad = nullptr, *m1 = nullptr, *m2 = nullptr, *w4b = nullptr;
    bf16 *W1b = nullptr, *W2b = nullptr, *W3b = nullptr, *W2t = nullptr, *W3t = nullptr;
    float* norm = nullptr;           // mu[35], sigma[35], y_scale
    float norm_h[2 * kIn + 1] = {};
    bf16 *Xb = nullptr, *Xbt = nullptr, *H1 = nullptr, *H1t = nullptr, *H2 = nullptr, *H2t = nullptr;
    bf16 *dZ3 = nullptr, *dZ3t = nullptr, *dZ2 = nullptr, *dZ2t = nullptr, *dZ1 = nullptr, *dZ1t = nullptr;
    float *Z1 = nullptr, *Z2 = nullptr, *Z3 = nullptr, *tb = nullptr, *loss = nullptr, *lr = nullptr;
    bf16 *I1 = nullptr, *I2 = nullptr;
    double* stats = nullptr;
    int* err = nullptr;
    long long step = 0;
    unsigned long long wait_ns = 2000000000ull;
    Maps mp;
    std::vector<void*> owned;
};

namespace {

pd_status mfail(pd_mlp* m, pd_status s, const std::string& msg)
{
    if (m) m->last = msg;
    return s;
}

#define MCUDA(m, call)                                                                          \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) return mfail(m, PD_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <typename T>
cudaError_t alloc(pd_mlp* m, T** p, size_t n)
{
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * std::max<size_t>(n, 1));
    if (e == cudaSuccess) {
        m->owned.push_back(*p);
        e = cudaMemsetAsync(*p, 0, sizeof(T) * std::max<size_t>(n, 1), m->stream);
    }
    return e;
}

GemmArgs base_args(pd_mlp* m, int M, int N, int K)
{
    GemmArgs a;
    std::memset(&a, 0, sizeof(a));
    a.M = M; a.N = N; a.K = K;
    a.chunks_per_split = (K + kBK - 1) / kBK;
    a.err = m->err;
    a.wait_ns = m->wait_ns;
    return a;
}

pd_status refresh_copies(pd_mlp* m)
{
    adam_kernel<<<(N_PARAM + 255) / 256, 256, 0, m->stream>>>(m->theta, m->grad, m->m1, m->m2, nullptr, 0.0f, 0.0f, 0.0f, 0,
                                                              m->W1b, m->W2b, m->W3b, m->W2t, m->W3t, m->w4b);
    MCUDA(m, cudaGetLastError());
    return PD_OK;
}

// forward and backward over the minibatch already in Xb / Xbt / tb
// (B rows, n_valid of them real); the gradient accumulates into m->grad
pd_status fwd_bwd(pd_mlp* m, int B, int n_valid)
{
    cudaStream_t st = m->stream;
    const float* th = m->theta;
    // forward: Z_l, H_l (row-major and transposed)
    {
        GemmArgs a = base_args(m, B, kWidth, kInCols);
        a.ldo = kWidth; a.ldt = m->cap; a.bias = th + OFF_B1; a.out_z = m->Z1; a.out_bf16 = m->H1; a.out_bf16_t = m->H1t;
        MCUDA(m, (launch_gemm<256, EPI_GELU>(m->mp.Xb, m->mp.W1, a, 1, st)));
    }
    {
        GemmArgs a = base_args(m, B, kWidth, kWidth);
        a.ldo = kWidth; a.ldt = m->cap; a.bias = th + OFF_B2; a.out_z = m->Z2; a.out_bf16 = m->H2; a.out_bf16_t = m->H2t;
        MCUDA(m, (launch_gemm<256, EPI_GELU>(m->mp.H1, m->mp.W2, a, 1, st)));
    }
    {
        GemmArgs a = base_args(m, B, kWidth, kWidth);
        a.ldo = kWidth; a.bias = th + OFF_B3; a.out_z = m->Z3;
        MCUDA(m, (launch_gemm<256, EPI_GELU>(m->mp.H2, m->mp.W3, a, 1, st)));
    }
    head_kernel<<<B / 32, 256, 0, st>>>(m->Z3, m->tb, m->w4b, m->theta, n_valid, m->cap, 1.0f / (float)n_valid,
                                        m->dZ3, m->dZ3t, m->grad, m->loss);
    MCUDA(m, cudaGetLastError());
    // split-K over the minibatch for the weight gradients
    const int kc = (B + kBK - 1) / kBK;
    const int per = std::max(1, (kc + 31) / 32);
    const int splits = (kc + per - 1) / per;
    {   // dW3 = dZ3^T H2
        GemmArgs a = base_args(m, kWidth, kWidth, B);
        a.ldo = kWidth; a.out_f32 = m->grad + OFF_W3; a.chunks_per_split = per;
        MCUDA(m, (launch_gemm<256, EPI_F32_ATOMIC, 4>(m->mp.dZ3t, m->mp.H2t, a, splits, st)));
    }
    {   // dZ2 = (dZ3 W3) g'(Z2)
        GemmArgs a = base_args(m, B, kWidth, kWidth);
        a.ldo = kWidth; a.ldt = m->cap; a.aux = m->Z2; a.out_bf16 = m->dZ2; a.out_bf16_t = m->dZ2t;
        MCUDA(m, (launch_gemm<256, EPI_GELU_BWD>(m->mp.dZ3, m->mp.W3t, a, 1, st)));
    }
    {   // dW2 = dZ2^T H1
        GemmArgs a = base_args(m, kWidth, kWidth, B);
        a.ldo = kWidth; a.out_f32 = m->grad + OFF_W2; a.chunks_per_split = per;
        MCUDA(m, (launch_gemm<256, EPI_F32_ATOMIC, 4>(m->mp.dZ2t, m->mp.H1t, a, splits, st)));
    }
    {   // dZ1 = (dZ2 W2) g'(Z1)
        GemmArgs a = base_args(m, B, kWidth, kWidth);
        a.ldo = kWidth; a.ldt = m->cap; a.aux = m->Z1; a.out_bf16 = m->dZ1; a.out_bf16_t = m->dZ1t;
        MCUDA(m, (launch_gemm<256, EPI_GELU_BWD>(m->mp.dZ2, m->mp.W2t, a, 1, st)));
    }
    {   // dW1 = dZ1^T X
        GemmArgs a = base_args(m, kWidth, kPad, B);
        a.ldo = kPad; a.out_f32 = m->grad + OFF_W1; a.chunks_per_split = per;
        MCUDA(m, (launch_gemm<64, EPI_F32_ATOMIC, 4>(m->mp.dZ1t, m->mp.Xbt, a, splits, st)));
    }
    bias_grad_kernel<<<dim3(kWidth, 3), 256, 0, st>>>(m->dZ1t, m->dZ2t, m->dZ3t, B, m->cap, m->grad);
    MCUDA(m, cudaGetLastError());
    return PD_OK;
}

pd_status check_err(pd_mlp* m)
{
    int h = 0;
    MCUDA(m, cudaMemcpyAsync(&h, m->err, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
    MCUDA(m, cudaStreamSynchronize(m->stream));
    if (h) {
        cudaMemsetAsync(m->err, 0, sizeof(int), m->stream);
        return mfail(m, PD_ETIMEOUT, "a tensor-core pipeline wait ran out of time");
    }
    return PD_OK;
}

}  // namespace

extern "C" {

pd_status pd_mlp_create(int max_batch, void* stream, pd_mlp** out)
{
    if (!out) return PD_EINVAL;
    *out = nullptr;
    if (max_batch < 128 || max_batch % 128 || max_batch > 65536) return PD_EINVAL;
    pd_mlp* m = new pd_mlp();
    cudaGetDevice(&m->device);
    m->stream = static_cast<cudaStream_t>(stream);
    m->cap = max_batch;
    cudaError_t e = get_encoder();
    if (e != cudaSuccess) { delete m; return PD_ECUDA; }
    const size_t B = (size_t)max_batch, C = (size_t)m->chunk, W = kWidth;
#define A_(p, n) if ((e = alloc(m, &m->p, (n))) != cudaSuccess) { pd_mlp_destroy(m); return PD_ENOMEM; }
    A_(theta, N_PARAM) A_(grad, N_PARAM) A_(m1, N_PARAM) A_(m2, N_PARAM) A_(w4b, W)
    A_(W1b, W * kInCols) A_(W2b, W * W) A_(W3b, W * W) A_(W2t, W * W) A_(W3t, W * W)
    A_(norm, 2 * kIn + 1) A_(Xb, B * kInCols) A_(Xbt, B * kPad) A_(H1, B * W) A_(H1t, B * W) A_(H2, B * W) A_(H2t, B * W)
    A_(dZ3, B * W) A_(dZ3t, B * W) A_(dZ2, B * W) A_(dZ2t, B * W) A_(dZ1, B * W) A_(dZ1t, B * W)
    A_(Z1, B * W) A_(Z2, B * W) A_(Z3, B * W) A_(tb, B) A_(loss, 1) A_(lr, 1) A_(I1, C * W) A_(I2, C * W)
    A_(stats, 2 * kIn + 1) A_(err, 1)
#undef A_
    Maps& p = m->mp;
    const long long b = max_batch;
    bool ok = make_map(&p.Xb, m->Xb, b, kInCols, kInCols, 128) && make_map(&p.W1, m->W1b, W, kInCols, kInCols, 256)
           && make_map(&p.H1, m->H1, b, W, W, 128) && make_map(&p.W2, m->W2b, W, W, W, 256)
           && make_map(&p.H2, m->H2, b, W, W, 128) && make_map(&p.W3, m->W3b, W, W, W, 256)
           && make_map(&p.dZ3t, m->dZ3t, W, max_batch, max_batch, 128) && make_map(&p.H2t, m->H2t, W, max_batch, max_batch, 256)
           && make_map(&p.dZ3, m->dZ3, b, W, W, 128) && make_map(&p.W3t, m->W3t, W, W, W, 256)
           && make_map(&p.dZ2t, m->dZ2t, W, max_batch, max_batch, 128) && make_map(&p.H1t, m->H1t, W, max_batch, max_batch, 256)
           && make_map(&p.dZ2, m->dZ2, b, W, W, 128) && make_map(&p.W2t, m->W2t, W, W, W, 256)
           && make_map(&p.dZ1t, m->dZ1t, W, max_batch, max_batch, 128) && make_map(&p.Xbt, m->Xbt, kPad, max_batch, max_batch, 64)
           && make_map(&p.I1, m->I1, C, W, W, 128) && make_map(&p.I2, m->I2, C, W, W, 128);
    if (!ok) { pd_mlp_destroy(m); return PD_ECUDA; }
    float nh[2 * kIn + 1];
    for (int k = 0; k < kIn; ++k) { nh[k] = 0.0f; nh[kIn + k] = 1.0f; }
    nh[2 * kIn] = 1.0f;
    std::memcpy(m->norm_h, nh, sizeof(nh));
    if (cudaMemcpyAsync(m->norm, nh, sizeof(nh), cudaMemcpyHostToDevice, m->stream) != cudaSuccess ||
        cudaStreamSynchronize(m->stream) != cudaSuccess) { pd_mlp_destroy(m); return PD_ECUDA; }
    *out = m;
    return PD_OK;
}

pd_status pd_mlp_destroy(pd_mlp* m)
{
    if (!m) return PD_EINVAL;
    if (m->stream) cudaStreamSynchronize(m->stream);
    for (void* p : m->owned) cudaFree(p);
    delete m;
    return PD_OK;
}

pd_status pd_mlp_set_stream(pd_mlp* m, void* stream)
{
    if (!m) return PD_EINVAL;
    m->stream = static_cast<cudaStream_t>(stream);
    return PD_OK;
}

pd_status pd_mlp_set_params(pd_mlp* m, const float* theta, int n)
{
    if (!m) return PD_EINVAL;
    if (!theta || n != N_PARAM) return mfail(m, PD_EINVAL, "expected PD_MLP_N_PARAM parameters");
    MCUDA(m, cudaMemcpyAsync(m->theta, theta, sizeof(float) * N_PARAM, cudaMemcpyHostToDevice, m->stream));
    MCUDA(m, cudaMemsetAsync(m->m1, 0, sizeof(float) * N_PARAM, m->stream));
    MCUDA(m, cudaMemsetAsync(m->m2, 0, sizeof(float) * N_PARAM, m->stream));
    MCUDA(m, cudaMemsetAsync(m->grad, 0, sizeof(float) * N_PARAM, m->stream));
    m->step = 0;
    pd_status rc = refresh_copies(m);
    if (rc) return rc;
    MCUDA(m, cudaStreamSynchronize(m->stream));
    return PD_OK;
}

pd_status pd_mlp_init(pd_mlp* m, unsigned long long seed)
{
    if (!m) return PD_EINVAL;
    init_kernel<<<(N_PARAM + 255) / 256, 256, 0, m->stream>>>(m->theta, seed);
    MCUDA(m, cudaGetLastError());
    MCUDA(m, cudaMemsetAsync(m->m1, 0, sizeof(float) * N_PARAM, m->stream));
    MCUDA(m, cudaMemsetAsync(m->m2, 0, sizeof(float) * N_PARAM, m->stream));
    MCUDA(m, cudaMemsetAsync(m->grad, 0, sizeof(float) * N_PARAM, m->stream));
    m->step = 0;
    return refresh_copies(m);
}

pd_status pd_mlp_get_params(pd_mlp* m, float* theta, int n)
{
    if (!m) return PD_EINVAL;
    if (!theta || n != N_PARAM) return mfail(m, PD_EINVAL, "expected PD_MLP_N_PARAM parameters");
    MCUDA(m, cudaMemcpyAsync(theta, m->theta, sizeof(float) * N_PARAM, cudaMemcpyDeviceToHost, m->stream));
    MCUDA(m, cudaStreamSynchronize(m->stream));
    return PD_OK;
}

pd_status pd_mlp_set_norm(pd_mlp* m, const float* mu, const float* sigma, float y_scale)
{
    if (!m) return PD_EINVAL;
    if (!mu || !sigma || !(y_scale > 0.0f)) return mfail(m, PD_EINVAL, "need mu, sigma and y_scale > 0");
    for (int k = 0; k < kIn; ++k) {
        if (!(sigma[k] > 0.0f)) return mfail(m, PD_EINVAL, "sigma must be positive");
        m->norm_h[k] = mu[k];
        m->norm_h[kIn + k] = sigma[k];
    }
    m->norm_h[2 * kIn] = y_scale;
    MCUDA(m, cudaMemcpyAsync(m->norm, m->norm_h, sizeof(m->norm_h), cudaMemcpyHostToDevice, m->stream));
    MCUDA(m, cudaStreamSynchronize(m->stream));
    return PD_OK;
}

pd_status pd_mlp_get_norm(pd_mlp* m, float* mu, float* sigma, float* y_scale)
{
    if (!m) return PD_EINVAL;
    for (int k = 0; k < kIn; ++k) {
        if (mu) mu[k] = m->norm_h[k];
        if (sigma) sigma[k] = m->norm_h[kIn + k];
    }
    if (y_scale) *y_scale = m->norm_h[2 * kIn];
    return PD_OK;
}

pd_status pd_mlp_fit_norm(pd_mlp* m, const float* X, const float* y, long long n)
{
    if (!m) return PD_EINVAL;
    if (!X || !y || n < 2) return mfail(m, PD_EINVAL, "need at least two rows");
    MCUDA(m, cudaMemsetAsync(m->stats, 0, sizeof(double) * (2 * kIn + 1), m->stream));
    norm_stats_kernel<<<304, 128, 0, m->stream>>>(X, y, n, m->stats);
    MCUDA(m, cudaGetLastError());
    double h[2 * kIn + 1];
    MCUDA(m, cudaMemcpyAsync(h, m->stats, sizeof(h), cudaMemcpyDeviceToHost, m->stream));
    MCUDA(m, cudaStreamSynchronize(m->stream));
    float mu[kIn], sg[kIn];
    for (int k = 0; k < kIn; ++k) {
        const double a = h[k] / n;
        const double v = std::max(0.0, h[kIn + 1 + k] / n - a * a);
        mu[k] = (float)a;
        sg[k] = v > 1e-24 ? (float)std::sqrt(v) : 1.0f;
    }
    const double ys = h[kIn] / n;
    return pd_mlp_set_norm(m, mu, sg, ys > 0 ? (float)ys : 1.0f);
}

pd_status pd_mlp_pack(pd_mlp* m, const float* X, const float* y, long long n, uint16_t* Xo, float* to)
{
    if (!m) return PD_EINVAL;
    if (n == 0) return PD_OK;
    if (!X || !Xo || n < 0) return mfail(m, PD_EINVAL, "null argument");
    const long long tot = n * kPad;
    pack_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, m->stream>>>(X, y, n, m->norm, reinterpret_cast<bf16*>(Xo), to);
    MCUDA(m, cudaGetLastError());
    return PD_OK;
}

pd_status pd_mlp_forward(pd_mlp* m, const uint16_t* X, long long n, float* y)
{
    pd::NvtxRange nvtx_range("pd_mlp_forward");
    if (!m) return PD_EINVAL;
    if (n == 0) return PD_OK;
    if (!X || !y || n < 0) return mfail(m, PD_EINVAL, "null argument");
    if ((n + 127) / 128 > (long long)INT32_MAX) return mfail(m, PD_EINVAL, "too many rows");
    CUtensorMap mx;
    if (!make_map(&mx, X, n, kInCols, kInCols, 128)) return mfail(m, PD_EINVAL, "input must be 16-byte aligned [n][128] BF16");
    static bool attr = false;
    if (!attr) {
        MCUDA(m, cudaFuncSetAttribute(mlp_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fused_smem_bytes()));
        attr = true;
    }
    int sms = 0;
    MCUDA(m, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device));
    FusedArgs a;
    a.n = n;
    a.n_tiles = (int)((n + 127) / 128);
    a.b1 = m->theta + OFF_B1;
    a.b2 = m->theta + OFF_B2;
    a.b3 = m->theta + OFF_B3;
    a.w4 = m->w4b;
    a.b4 = m->theta + OFF_B4;
    a.y = y;
    a.err = m->err;
    a.wait_ns = m->wait_ns;
    const int grid = std::min(a.n_tiles, std::max(1, sms));
    mlp_fused_kernel<<<grid, kFThreads, fused_smem_bytes(), m->stream>>>(mx, m->mp.W1, m->mp.W2, m->mp.W3, a);
    MCUDA(m, cudaGetLastError());
    return PD_OK;
}

pd_status pd_mlp_gradient(pd_mlp* m, const uint16_t* X, const float* t, int n, float* grad_out, float* loss_host)
{
    if (!m) return PD_EINVAL;
    if (!X || !t || n < 1 || n > m->cap) return mfail(m, PD_EINVAL, "need 1 <= n <= max_batch rows");
    const int B = (n + 127) / 128 * 128;
    cudaStream_t st = m->stream;
    MCUDA(m, cudaMemsetAsync(m->grad, 0, sizeof(float) * N_PARAM, st));
    MCUDA(m, cudaMemsetAsync(m->loss, 0, sizeof(float), st));
    gather_kernel<<<B / 64, 256, 0, st>>>(reinterpret_cast<const bf16*>(X), t, n, 0ull, 0ull, 0, n, m->cap, m->Xb, m->Xbt, m->tb);
    MCUDA(m, cudaGetLastError());
    pd_status rc = fwd_bwd(m, B, n);
    if (rc) return rc;
    if (grad_out) MCUDA(m, cudaMemcpyAsync(grad_out, m->grad, sizeof(float) * N_PARAM, cudaMemcpyDeviceToDevice, st));
    if (loss_host) {
        float h = 0.0f;
        MCUDA(m, cudaMemcpyAsync(&h, m->loss, sizeof(float), cudaMemcpyDeviceToHost, st));
        rc = check_err(m);
        if (rc) return rc;
        *loss_host = h / (float)n;
    }
    return PD_OK;
}

pd_status pd_mlp_adam_step(pd_mlp* m, float lr)
{
    if (!m) return PD_EINVAL;
    m->step += 1;
    const float c1 = (float)(1.0 / (1.0 - std::pow(0.9, (double)m->step)));
    const float c2 = (float)(1.0 / (1.0 - std::pow(0.999, (double)m->step)));
    adam_kernel<<<(N_PARAM + 255) / 256, 256, 0, m->stream>>>(m->theta, m->grad, m->m1, m->m2, nullptr, lr, c1, c2, 1,
                                                              m->W1b, m->W2b, m->W3b, m->W2t, m->W3t, m->w4b);
    MCUDA(m, cudaGetLastError());
    return PD_OK;
}

pd_status pd_mlp_train(pd_mlp* m, const uint16_t* X, const float* T, long long n, int batch, int epochs, float lr_max,
                       unsigned long long seed, float* loss_hist)
{
    pd::NvtxRange nvtx_range("pd_mlp_train");
    if (!m) return PD_EINVAL;
    if (!X || !T) return mfail(m, PD_EINVAL, "null argument");
    if (batch < 128 || batch % 128 || batch > m->cap) return mfail(m, PD_EINVAL, "batch must be a multiple of 128 and <= max_batch");
    if (n < batch || epochs < 0 || !(lr_max > 0.0f)) return mfail(m, PD_EINVAL, "need n >= batch, epochs >= 0, lr_max > 0");
    cudaStream_t st = m->stream;
    const long long spe = n / batch;
    const long long total = spe * (long long)epochs;
    unsigned long long rs = seed ^ 0x9E3779B97F4A7C15ull;
    auto next = [&rs]() {   // splitmix64
        unsigned long long z = (rs += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    long long g = 0;
    for (int e = 0; e < epochs; ++e) {
        unsigned long long a = 1 + next() % (unsigned long long)(n - 1 > 0 ? n - 1 : 1);
        while (std::gcd(a, (unsigned long long)n) != 1ull) a = 1 + (a % (unsigned long long)n);
        const unsigned long long b = next() % (unsigned long long)n;
        MCUDA(m, cudaMemsetAsync(m->loss, 0, sizeof(float), st));
        for (long long s = 0; s < spe; ++s, ++g) {
            lr_kernel<<<1, 1, 0, st>>>(m->lr, g, total, lr_max);
            gather_kernel<<<batch / 64, 256, 0, st>>>(reinterpret_cast<const bf16*>(X), T, n, a, b, s * batch, batch, m->cap,
                                                      m->Xb, m->Xbt, m->tb);
            MCUDA(m, cudaGetLastError());
            pd_status rc = fwd_bwd(m, batch, batch);
            if (rc) return rc;
            m->step += 1;
            const float c1 = (float)(1.0 / (1.0 - std::pow(0.9, (double)m->step)));
            const float c2 = (float)(1.0 / (1.0 - std::pow(0.999, (double)m->step)));
            adam_kernel<<<(N_PARAM + 255) / 256, 256, 0, st>>>(m->theta, m->grad, m->m1, m->m2, m->lr, 0.0f, c1, c2, 1,
                                                               m->W1b, m->W2b, m->W3b, m->W2t, m->W3t, m->w4b);
            MCUDA(m, cudaGetLastError());
        }
        if (loss_hist) {
            float h = 0.0f;
            MCUDA(m, cudaMemcpyAsync(&h, m->loss, sizeof(float), cudaMemcpyDeviceToHost, st));
            MCUDA(m, cudaStreamSynchronize(st));
            loss_hist[e] = h / (float)(spe * batch);
        }
    }
    return check_err(m);
}

pd_status pd_mlp_sync(pd_mlp* m)
{
    if (!m) return PD_EINVAL;
    return check_err(m);
}

const char* pd_mlp_last_error(const pd_mlp* m)
{
    return m ? m->last.c_str() : "null network";
}

}  // extern "C"

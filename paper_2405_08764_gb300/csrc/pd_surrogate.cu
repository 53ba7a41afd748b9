// The surrogate on a grid: per-patch features from the macro field, the
// residual check against a one-micro-step burst, the fallback of the failing
// patches (a compacted list) to the full burst, and the macro update (C ABI of
// include/pd_surrogate.h).
#include "pd_internal.h"
#include "pd_surrogate.h"

#include <cuda_bf16.h>

#include <cmath>
#include <string>

using namespace pd;

namespace {

constexpr int kIn = PD_MLP_N_IN;
constexpr int kPad = PD_MLP_N_PAD;
constexpr int kInCols = PD_MLP_IN_COLS;
constexpr int kStatic = 10;

__device__ __forceinline__ void diff_basis(const double u[5], double e[5])
{
    // offsets -2..2 -> value, first, second, third and fourth differences, from
    // the mirrored sums p_k and differences m_k (nine FP64 operations, not twelve)
    const double p1 = u[3] + u[1], p2 = u[4] + u[0];
    const double m1 = u[3] - u[1], m2 = u[4] - u[0];
    e[0] = u[2];
    e[1] = 0.5 * m1;
    e[2] = fma(-2.0, u[2], p1);
    e[3] = fma(0.5, m2, -m1);
    e[4] = fma(6.0, u[2], fma(-4.0, p1, p2));
}

// One patch per thread: the 5x5 stencil (xi wraps on periodic grids, clamps
// otherwise; eta clamps), its difference basis normalised by s, the metric
// terms times the matching differences, the coefficient samples; then the
// network input row (high and low BF16 parts of the standardised features)
// and the output scale and/or the raw features and R s.
__global__ void features_kernel(const InstDev I, const double* __restrict__ U, const float* __restrict__ stat,
                                const double* __restrict__ R, const float* __restrict__ norm,
                                __nv_bfloat16* __restrict__ X, double* __restrict__ scale,
                                float* __restrict__ Xraw, double* __restrict__ Rs,
                                const double* __restrict__ T1, const double* __restrict__ sT, double* __restrict__ F1)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= I.n_patch) return;
    const int i = I.i0 + p % I.ncols, j = 1 + p / I.ncols;
    double raw[5][5], a[5][5];
    for (int q = 0; q < 5; ++q) {
        const int row = min(max(j + q - 2, 0), I.n_eta);
        for (int o = 0; o < 5; ++o) {
            int c = i + o - 2;
            if (I.periodic) c = (c % I.nxp + I.nxp) % I.nxp;
            else c = min(max(c, 0), I.n_xi);
            raw[q][o] = U[(long long)row * I.nxp + c];
        }
        diff_basis(raw[q], a[q]);
    }
    if (F1) {
        // the check estimate from the 3x3 stencil (rows j-1..j+1 and columns
        // i-1..i+1 are never clamped for a patch) and the one-step basis
        const double* t = T1 + (long long)p * 10;
        double f = *sT * t[9];
        for (int pp = -1; pp <= 1; ++pp)
            for (int qq = -1; qq <= 1; ++qq) f = fma(t[(pp + 1) * 3 + qq + 1], raw[qq + 2][pp + 2], f);
        F1[p] = f;
    }
    double D[25];
    for (int po = 0; po < 5; ++po) {
        double u[5], e[5];
        for (int q = 0; q < 5; ++q) u[q] = a[q][po];
        diff_basis(u, e);
        for (int qo = 0; qo < 5; ++qo) D[5 * qo + po] = e[qo];
    }
    // s = max |D[k]| (k >= 1) exactly, compared as integers: for doubles with the
    // sign bit cleared the bit patterns order like the magnitudes (FP64
    // comparisons would issue on the slow FP64 pipe)
    unsigned long long sb = 0ull;
    for (int k = 1; k < 25; ++k) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(D[k]) & 0x7fffffffffffffffull;
        sb = b > sb ? b : sb;
    }
    const double s = __longlong_as_double((long long)sb);
    float x[kIn];
    // the normalised features need FP32 precision only: FP32 quotients
    const float sf = (float)s, d0 = (float)D[0];
    const float den = fabsf(d0) + sf;
    x[0] = den > 0.0f ? d0 / den : 0.0f;
    const float inv_s = sf > 0.0f ? 1.0f / sf : 0.0f;
    for (int k = 1; k < 25; ++k) x[k] = (float)D[k] * inv_s;
    const float* st = stat + (long long)p * kStatic;
    x[25] = st[0] * x[2];
    x[26] = st[1] * x[10];
    x[27] = st[2] * x[1];
    x[28] = st[3] * x[5];
    for (int k = 4; k < kStatic; ++k) x[25 + k] = st[k];
    const double rs = R[p] * s;
    if (Xraw) {
        for (int k = 0; k < kIn; ++k) Xraw[(long long)p * kIn + k] = x[k];
    }
    if (Rs) Rs[p] = rs;
    if (X) {
        __nv_bfloat162* hi = reinterpret_cast<__nv_bfloat162*>(X + (long long)p * kInCols);
        __nv_bfloat162* lo = hi + kPad / 2;
        for (int k = 0; k < kPad; k += 2) {
            const float v0 = k < kIn ? (x[k] - norm[k]) / norm[kIn + k] : 0.0f;
            const float v1 = k + 1 < kIn ? (x[k + 1] - norm[k + 1]) / norm[kIn + k + 1] : 0.0f;
            const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
            hi[k / 2] = h;
            lo[k / 2] = __floats2bfloat162_rn(v0 - __bfloat162float(h.x), v1 - __bfloat162float(h.y));
        }
    }
    if (scale) scale[p] = rs * (double)norm[2 * kIn];
}

__global__ void targets_kernel(int n, const double* __restrict__ dU, const double* __restrict__ Rs, double tau,
                               float* __restrict__ y)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const double r = Rs[p];
    y[p] = r > 0.0 ? (float)(dU[p] / (tau * r)) : 0.0f;
}

__global__ void scale_out_kernel(int n, const double* __restrict__ in, double f, double* __restrict__ out)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) out[p] = in[p] * f;
}

__global__ void predict_kernel(int n, const float* __restrict__ yhat, const double* __restrict__ scale,
                               double* __restrict__ out)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) out[p] = (double)yhat[p] * scale[p];
}

// sum over patches of F1^2
__global__ void sumsq_kernel(int n, const double* __restrict__ F1, double* __restrict__ acc)
{
    double v = 0.0;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const double f = F1[p];
        v += f * f;
    }
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __shared__ double red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        atomicAdd(acc, t);
    }
}

// The residual check: keep F_hat = yhat * scale when |F_hat - F1| <= eps (|F1| + rho),
// rho = sqrt(sum F1^2 / n), writing its restricted change F_hat tau; append the
// other patches to the fallback list.
// One thread per patch, 256 per block: the RMS floor once per block, the
// fallback patches of the block packed by warp ballots and one pair of atomics
// per block (a single counter for every warp of the grid was the bottleneck)
__global__ void __launch_bounds__(256)
check_kernel(int n, const float* __restrict__ yhat, const double* __restrict__ scale,
             const double* __restrict__ F1v, const double* __restrict__ sumsq, double tau, double eps,
             double* __restrict__ dUf, int* __restrict__ list, int* __restrict__ list_n,
             unsigned long long* __restrict__ n_fb)
{
    __shared__ double rho_s;
    __shared__ int cnt_s[8], base_s;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) rho_s = sqrt(*sumsq / (double)n);
    __syncthreads();
    bool fb = false;
    if (p < n) {
        const double rho = rho_s;
        const double F1 = F1v[p];
        const double Fh = (double)yhat[p] * scale[p];
        const bool ok = eps >= 0.0 && isfinite(Fh) && fabs(Fh - F1) <= eps * (fabs(F1) + rho);
        if (ok) dUf[p] = Fh * tau;
        fb = !ok;
    }
    const unsigned b = __ballot_sync(0xffffffffu, fb);
    if (lane == 0) cnt_s[warp] = __popc(b);
    __syncthreads();
    if (threadIdx.x == 0) {
        int tot = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            const int c = cnt_s[w];
            cnt_s[w] = tot;
            tot += c;
        }
        base_s = tot ? atomicAdd(list_n, tot) : 0;
        if (tot) atomicAdd(n_fb, (unsigned long long)tot);
    }
    __syncthreads();
    if (fb) list[base_s + cnt_s[warp] + __popc(b & ((1u << lane) - 1u))] = p;
}

// The scheme with bursts of one micro step (tau = dt): per patch the restricted
// change of one forward-Euler step from the lift, exactly the check's estimate
// F1 = sum_q T1_q U_q + s(T) T1_9 over the 3x3 stencil (never clamped for a
// patch), written as dU = F1 tau, the change the projection divides by tau.
// One patch per thread.
__global__ void f1_step_kernel(const InstDev I, const double* __restrict__ U, const double* __restrict__ T1,
                               const double* __restrict__ sT, double tau, double* __restrict__ dU)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= I.n_patch) return;
    const int i = I.i0 + p % I.ncols, j = 1 + p / I.ncols;
    const double* t = T1 + (long long)p * 10;
    double f = *sT * t[9];
    for (int pp = -1; pp <= 1; ++pp) {
        int c = i + pp;
        if (I.periodic) c = c < 0 ? c + I.nxp : (c >= I.nxp ? c - I.nxp : c);
        for (int qq = -1; qq <= 1; ++qq) f = fma(t[(pp + 1) * 3 + qq + 1], U[(long long)(j + qq) * I.nxp + c], f);
    }
    dU[p] = f * tau;
}

__global__ void maxabs_kernel(long long n, const double* __restrict__ U, unsigned long long* __restrict__ out)
{
    double v = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        v = fmax(v, fabs(U[k]));
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    // non-negative doubles order like their bit patterns
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ double uniform01(unsigned long long z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return ((double)(z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

__global__ void perturb_kernel(const InstDev I, const double* __restrict__ U, const unsigned long long* __restrict__ mx,
                               double rel_sigma, unsigned long long seed, double* __restrict__ V)
{
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long n = (long long)I.nxp * I.nyp;
    if (k >= n) return;
    const int j = (int)(k / I.nxp), i = (int)(k - (long long)j * I.nxp);
    const bool interior = j > 0 && j < I.n_eta && (I.periodic || (i > 0 && i < I.n_xi));
    double v = U[k];
    if (interior) {
        const double u1 = uniform01(seed + 2 * (unsigned long long)k * 0x9E3779B97F4A7C15ull);
        const double u2 = uniform01(seed + (2 * (unsigned long long)k + 1) * 0x9E3779B97F4A7C15ull);
        const double z = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
        v += rel_sigma * __longlong_as_double((long long)*mx) * z;
    }
    V[k] = v;
}

}  // namespace

struct pd_surrogate {
    pd_grid* g = nullptr;
    pd_mlp* m = nullptr;
    GridAccess ga;
    int n = 0;
    float* stat = nullptr;
    double* R = nullptr;
    uint16_t* X = nullptr;
    double *scale = nullptr, *F1 = nullptr, *dUf = nullptr, *sumsq = nullptr, *T1 = nullptr;
    float* yhat = nullptr;
    float* norm = nullptr;
    int *list = nullptr, *list_n = nullptr;
    unsigned long long* n_fb = nullptr;
    unsigned long long* umax = nullptr;
    double* tabK = nullptr;
    size_t tab_steps = 0;
    long long patch_steps = 0;
    std::string last;
};

namespace {

pd_status sfail(pd_surrogate* s, pd_status rc, const std::string& msg)
{
    if (s) {
        s->last = msg;
        grid_message(s->g, msg.c_str());
    }
    return rc;
}

#define SCUDA(s, call)                                                                                      \
    do {                                                                                                    \
        cudaError_t e_ = (call);                                                                            \
        if (e_ != cudaSuccess) return sfail(s, PD_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

pd_status upload_norm(pd_surrogate* s)
{
    float h[2 * kIn + 1];
    pd_status rc = pd_mlp_get_norm(s->m, h, h + kIn, h + 2 * kIn);
    if (rc) return sfail(s, rc, "network normalisation");
    SCUDA(s, cudaMemcpyAsync(s->norm, h, sizeof(h), cudaMemcpyHostToDevice, s->ga.stream));
    SCUDA(s, cudaStreamSynchronize(s->ga.stream));
    return PD_OK;
}

pd_status ensure_tables(pd_surrogate* s, int n_steps)
{
    if ((size_t)n_steps <= s->tab_steps) return PD_OK;
    SCUDA(s, cudaStreamSynchronize(s->ga.stream));
    cudaFree(s->tabK);
    s->tabK = nullptr;
    SCUDA(s, cudaMalloc(&s->tabK, sizeof(double) * (size_t)n_steps * (s->ga.I.K + kTabExtra)));
    s->tab_steps = (size_t)n_steps;
    return PD_OK;
}

unsigned blocks(int n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

extern "C" {

pd_status pd_surrogate_create(pd_grid* g, pd_mlp* m, pd_surrogate** out)
{
    if (!g || !m || !out) return PD_EINVAL;
    *out = nullptr;
    pd_surrogate* s = new pd_surrogate();
    s->g = g;
    s->m = m;
    pd_status rc = grid_access(g, 0, s->ga);
    if (rc) { delete s; return rc; }
    const InstDev& I = s->ga.I;
    if (s->ga.n_inst != 1) { delete s; grid_message(g, "the surrogate takes a grid of one instance"); return PD_EINVAL; }
    if (I.coef_mode != COEF_RECORDS || !fused_supported(I) || I.restrict_mode != PD_RESTRICT_LIFTED
        || I.micro != PD_MICRO_FE) {
        delete s;
        grid_message(g, "the surrogate needs per-point coefficient records, m_xi == m_eta in {3,5,7,9,11}, the "
                        "lifted restriction and forward-Euler micro steps");
        return PD_EINVAL;
    }
    s->n = I.n_patch;
    const size_t n = (size_t)s->n;
    cudaError_t e = cudaSuccess;
    auto A = [&](void** p, size_t bytes) { if (e == cudaSuccess) e = cudaMalloc(p, bytes); };
    A((void**)&s->stat, n * kStatic * sizeof(float));
    A((void**)&s->R, n * sizeof(double));
    A((void**)&s->X, n * kInCols * sizeof(uint16_t));
    A((void**)&s->scale, n * sizeof(double));
    A((void**)&s->F1, n * sizeof(double));
    A((void**)&s->T1, n * 10 * sizeof(double));
    A((void**)&s->dUf, n * sizeof(double));
    A((void**)&s->yhat, n * sizeof(float));
    A((void**)&s->list, n * sizeof(int));
    A((void**)&s->list_n, sizeof(int));
    A((void**)&s->sumsq, sizeof(double));
    A((void**)&s->norm, (2 * kIn + 1) * sizeof(float));
    A((void**)&s->n_fb, sizeof(unsigned long long));
    A((void**)&s->umax, sizeof(unsigned long long));
    if (e != cudaSuccess) { pd_surrogate_destroy(s); grid_message(g, "surrogate buffers"); return PD_ENOMEM; }
    cudaStream_t st = s->ga.stream;
    e = cudaMemsetAsync(s->n_fb, 0, sizeof(unsigned long long), st);
    const double tau = I.K * I.dt;
    if (e == cudaSuccess) e = launch_surrogate_static(I, s->ga.coef, tau, s->stat, s->R, st);
    if (e == cudaSuccess) e = launch_one_step_basis(I, s->ga.prec, s->T1, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        grid_message(g, cudaGetErrorString(e));
        pd_surrogate_destroy(s);
        return PD_ECUDA;
    }
    grid_count_launches(g, 2);
    *out = s;
    return PD_OK;
}

pd_status pd_surrogate_destroy(pd_surrogate* s)
{
    if (!s) return PD_EINVAL;
    if (s->ga.stream) cudaStreamSynchronize(s->ga.stream);
    void* ptrs[] = { s->stat, s->R, s->X, s->scale, s->F1, s->T1, s->dUf, s->yhat, s->list, s->list_n, s->sumsq,
                     s->norm, s->n_fb, s->umax, s->tabK };
    for (void* p : ptrs) cudaFree(p);
    delete s;
    return PD_OK;
}

pd_status pd_surrogate_features(pd_surrogate* s, const double* U, uint16_t* X, double* scale, float* Xraw, double* Rs)
{
    NvtxRange nvtx_range("pd_surrogate_features");
    if (!s) return PD_EINVAL;
    if (!U) return sfail(s, PD_EINVAL, "null field");
    if (X || scale) {
        pd_status rc = upload_norm(s);
        if (rc) return rc;
    }
    features_kernel<<<blocks(s->n, 128), 128, 0, s->ga.stream>>>(s->ga.I, U, s->stat, s->R, s->norm,
                                                                 reinterpret_cast<__nv_bfloat16*>(X), scale, Xraw, Rs,
                                                                 nullptr, nullptr, nullptr);
    SCUDA(s, cudaGetLastError());
    grid_count_launches(s->g, 1);
    return PD_OK;
}

pd_status pd_surrogate_targets(pd_surrogate* s, const double* U, double t, const double* Rs, float* y)
{
    NvtxRange nvtx_range("pd_surrogate_targets");
    if (!s) return PD_EINVAL;
    if (!U || !Rs || !y) return sfail(s, PD_EINVAL, "null argument");
    pd_status rc = ensure_tables(s, 1);
    if (rc) return rc;
    const InstDev& I = s->ga.I;
    cudaStream_t st = s->ga.stream;
    SCUDA(s, launch_time_table(I, t, 1.0, 1, s->tabK, st));
    SCUDA(s, launch_patch_dU(I, s->ga.prec, U, s->tabK, I.K, s->dUf, nullptr, nullptr, st));
    targets_kernel<<<blocks(s->n, 256), 256, 0, st>>>(s->n, s->dUf, Rs, I.K * I.dt, y);
    SCUDA(s, cudaGetLastError());
    grid_count_launches(s->g, 3);
    return PD_OK;
}

pd_status pd_surrogate_evaluate(pd_surrogate* s, const double* U, double t, double* F_hat, double* F1, double* F)
{
    NvtxRange nvtx_range("pd_surrogate_evaluate");
    if (!s) return PD_EINVAL;
    if (!U) return sfail(s, PD_EINVAL, "null field");
    pd_status rc = ensure_tables(s, 1);
    if (rc) return rc;
    rc = upload_norm(s);
    if (rc) return rc;
    const InstDev& I = s->ga.I;
    cudaStream_t st = s->ga.stream;
    SCUDA(s, launch_time_table(I, t, 1.0, 1, s->tabK, st));
    features_kernel<<<blocks(s->n, 128), 128, 0, st>>>(I, U, s->stat, s->R, s->norm,
                                                       reinterpret_cast<__nv_bfloat16*>(s->X), s->scale, nullptr, nullptr,
                                                       s->T1, s->tabK + I.K, s->F1);
    SCUDA(s, cudaGetLastError());
    if (F_hat) {
        pd_mlp_set_stream(s->m, st);
        rc = pd_mlp_forward(s->m, s->X, s->n, s->yhat);
        if (rc) return sfail(s, rc, pd_mlp_last_error(s->m));
        predict_kernel<<<blocks(s->n, 256), 256, 0, st>>>(s->n, s->yhat, s->scale, F_hat);
        SCUDA(s, cudaGetLastError());
    }
    if (F1) SCUDA(s, cudaMemcpyAsync(F1, s->F1, sizeof(double) * s->n, cudaMemcpyDeviceToDevice, st));
    if (F) {
        SCUDA(s, launch_patch_dU(I, s->ga.prec, U, s->tabK, I.K, s->dUf, nullptr, nullptr, st));
        scale_out_kernel<<<blocks(s->n, 256), 256, 0, st>>>(s->n, s->dUf, 1.0 / (I.K * I.dt), F);
        SCUDA(s, cudaGetLastError());
    }
    return PD_OK;
}

pd_status pd_surrogate_step(pd_surrogate* s, double* U, double t0, double dt_macro, int n_macro, double eps)
{
    NvtxRange nvtx_range("pd_surrogate_step");
    if (!s) return PD_EINVAL;
    if (!U || n_macro < 0) return sfail(s, PD_EINVAL, "null field or negative step count");
    if (n_macro == 0) return PD_OK;
    pd_status rc = upload_norm(s);
    if (rc) return rc;
    rc = ensure_tables(s, n_macro);
    if (rc) return rc;
    const InstDev& I = s->ga.I;
    cudaStream_t st = s->ga.stream;
    const double dtm = dt_macro > 0 ? dt_macro : s->ga.dtm_sugg;
    const double tau = I.K * I.dt;
    const int strideK = I.K + kTabExtra;
    SCUDA(s, launch_time_table(I, t0, dtm, n_macro, s->tabK, st));
    pd_mlp_set_stream(s->m, st);
    long long nl = 1;
    for (int k = 0; k < n_macro; ++k) {
        const double t = t0 + k * dtm;
        const double* row = s->tabK + (size_t)k * strideK;
        features_kernel<<<blocks(s->n, 128), 128, 0, st>>>(I, U, s->stat, s->R, s->norm,
                                                           reinterpret_cast<__nv_bfloat16*>(s->X), s->scale, nullptr, nullptr,
                                                           s->T1, row + I.K, s->F1);
        SCUDA(s, cudaGetLastError());
        rc = pd_mlp_forward(s->m, s->X, s->n, s->yhat);
        if (rc) return sfail(s, rc, pd_mlp_last_error(s->m));
        SCUDA(s, cudaMemsetAsync(s->sumsq, 0, sizeof(double), st));
        SCUDA(s, cudaMemsetAsync(s->list_n, 0, sizeof(int), st));
        sumsq_kernel<<<304, 256, 0, st>>>(s->n, s->F1, s->sumsq);
        check_kernel<<<blocks(s->n, 256), 256, 0, st>>>(s->n, s->yhat, s->scale, s->F1, s->sumsq, tau, eps, s->dUf,
                                                        s->list, s->list_n, s->n_fb);
        SCUDA(s, cudaGetLastError());
        SCUDA(s, launch_patch_dU(I, s->ga.prec, U, row, I.K, s->dUf, s->list, s->list_n, st));
        SCUDA(s, launch_project(I, U, s->dUf, t, dtm, st));
        nl += 6 + 3 * ((s->n + 65535) / 65536);
    }
    grid_count_launches(s->g, nl);
    s->patch_steps += (long long)s->n * n_macro;
    return PD_OK;
}

pd_status pd_surrogate_step_f1(pd_surrogate* s, double* U, double t0, double dt_macro, int n_macro)
{
    NvtxRange nvtx_range("pd_surrogate_step_f1");
    if (!s) return PD_EINVAL;
    if (!U || n_macro < 0) return sfail(s, PD_EINVAL, "null field or negative step count");
    if (n_macro == 0) return PD_OK;
    pd_status rc = ensure_tables(s, n_macro);
    if (rc) return rc;
    const InstDev& I = s->ga.I;
    cudaStream_t st = s->ga.stream;
    const double dtm = dt_macro > 0 ? dt_macro : s->ga.dtm_sugg;
    const int strideK = I.K + kTabExtra;
    SCUDA(s, launch_time_table(I, t0, dtm, n_macro, s->tabK, st));
    for (int k = 0; k < n_macro; ++k) {
        const double t = t0 + k * dtm;
        const double* row = s->tabK + (size_t)k * strideK;
        f1_step_kernel<<<blocks(s->n, 128), 128, 0, st>>>(I, U, s->T1, row + I.K, I.K * I.dt, s->dUf);
        SCUDA(s, cudaGetLastError());
        SCUDA(s, launch_project(I, U, s->dUf, t, dtm, st));
    }
    grid_count_launches(s->g, 1 + 2LL * n_macro);
    return PD_OK;
}

pd_status pd_surrogate_perturb(pd_surrogate* s, const double* U, double rel_sigma, unsigned long long seed, double* V)
{
    if (!s) return PD_EINVAL;
    if (!U || !V || !(rel_sigma >= 0.0)) return sfail(s, PD_EINVAL, "null field or negative sigma");
    const InstDev& I = s->ga.I;
    const long long n = (long long)I.nxp * I.nyp;
    cudaStream_t st = s->ga.stream;
    SCUDA(s, cudaMemsetAsync(s->umax, 0, sizeof(unsigned long long), st));
    maxabs_kernel<<<304, 256, 0, st>>>(n, U, s->umax);
    perturb_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(I, U, s->umax, rel_sigma, seed, V);
    SCUDA(s, cudaGetLastError());
    grid_count_launches(s->g, 2);
    return PD_OK;
}

pd_status pd_surrogate_counts(pd_surrogate* s, long long* patch_steps, long long* fallbacks)
{
    if (!s) return PD_EINVAL;
    unsigned long long h = 0;
    SCUDA(s, cudaMemcpyAsync(&h, s->n_fb, sizeof(h), cudaMemcpyDeviceToHost, s->ga.stream));
    SCUDA(s, cudaStreamSynchronize(s->ga.stream));
    if (patch_steps) *patch_steps = s->patch_steps;
    if (fallbacks) *fallbacks = (long long)h;
    return PD_OK;
}

}  // extern "C"

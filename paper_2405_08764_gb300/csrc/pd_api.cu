// Host side of libpd: descriptors, device buffers, setup, launch sequencing,
// CUDA-graph capture of the macro loop, checkpoints and error reporting.
#include "pd_internal.h"

#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <map>
#include <string>
#include <utility>
#include <vector>

using namespace pd;

namespace {

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// header block of the micro-state buffer: lift time, s(t), burst time table
constexpr size_t kStateHeader = 256 + 8 * (size_t)kMaxK + 256;

struct Inst {
    pd_grid_desc d;
    InstDev I;                       // host copy (pointers are device pointers)
    void* rec = nullptr;             // coefficient records
    void* brec = nullptr;            // burst records (weights, source, forcing basis)
    void* arec_c = nullptr;          // ADI line records (eta lines, xi lines)
    void* arec_r = nullptr;
    int2* bnd_ij = nullptr;
    double2* bnd_xy = nullptr;
    double* amp = nullptr;
    pd_coeff_desc coef;
    bool coef_set = false;
    double dt = 0, tau = 0, dtm_sugg = 0;
    std::vector<int2> bnd_host;
    double* col_tab = nullptr;       // table coefficient mode
    double* row_tab = nullptr;
    float* col_tab_f = nullptr;      // FP32 copies
    float* row_tab_f = nullptr;
    int* bnd_off = nullptr;          // boundary nodes owned by each item warp (persistent kernel)
    int* bnd_idx = nullptr;
    int n_item = 0;
};

struct GraphEntry {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int n_nodes = 0;
};

struct GraphKey {
    uintptr_t U;
    int n;
    std::vector<double> dtm;
    bool operator<(const GraphKey& o) const
    {
        if (U != o.U) return U < o.U;
        if (n != o.n) return n < o.n;
        return dtm < o.dtm;
    }
};

}  // namespace

struct pd_grid {
    std::vector<Inst> inst;
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;
    int* err = nullptr;              // device error flags
    unsigned long long* acc = nullptr; // device accumulators (3)
    double* U_scratch = nullptr;     // second macro buffer for pd_step
    size_t U_scratch_n = 0;
    double* tab = nullptr;           // time tables (pd_step)
    size_t tab_n = 0;
    char* state = nullptr;           // internal micro state (fallback step path)
    double* dU = nullptr;
    long long n_macro_total = 0, n_patch_total = 0;
    size_t state_bytes = 0;
    bool graphs = true;
    std::map<GraphKey, GraphEntry> gcache;
    long long launches = 0;
    std::string last;
    int device = 0;
    bool timing = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> tev;   // pending event pairs
    std::vector<cudaEvent_t> tfree;
    double t_ms = 0.0;
    long long t_launches = 0;
    int* flags = nullptr;            // per-item-warp step counters (persistent kernel)
    size_t flags_n = 0;
    bool persist = true;
    int integrator = PD_INT_EULER;   // outer (projective) integrator of pd_step
    int q_refresh = 1;               // edge-data refreshes per burst
    double* Dq = nullptr;            // refresh increment field (macro-sized)
    double* dRa = nullptr;           // restricted changes so far (refresh)
    double* dRb = nullptr;
    double* dRz = nullptr;           // zeros (no reference bias)
    double* S2 = nullptr;            // second scratch field (Heun)
    double* dUa = nullptr;           // per-patch restricted changes (AB2 history)
    double* dUb = nullptr;
    long long wait_ns = 250000000LL;
    int silent_warp = -1;
    // batched execution (many instances or table-mode coefficients)
    int storage = 0;                 // 0 auto, 1 records, 2 tables
    InstDev* insts_dev = nullptr;
    BatchItem* items_dev = nullptr;
    int n_items = 0;
    // classes of the batch: items [cls_beg[c], cls_beg[c] + cls_n[c]) are the
    // patch groups of the separable-map instances with m = cls_m[c] (cls_sep[c],
    // FP32 grids), or the patch groups of the other instances and the boundary
    // chunks of all instances with m = cls_m[c]
    std::vector<int> cls_m, cls_beg, cls_n;
    std::vector<char> cls_sep;
    bool batch_dirty = true;
    double* dtm_dev = nullptr;
    double2* scale_dev = nullptr;    // per instance (dtm inv_tau inv_nn, dtm inv_tau)
    std::vector<double> dtm_host;
    long long* tab_off_dev = nullptr;
    int* counters = nullptr;
    size_t counters_n = 0;
    int bt_block = 128;
    bool bt_half = false;
    bool bt_tuned = false;
    bool autotune = true;
    std::vector<double> tune_log;   // ms per macro step of each candidate
};

namespace {

pd_status fail(pd_grid* g, pd_status s, const std::string& msg)
{
    if (g) g->last = msg;
    return s;
}

pd_status cuda_fail(pd_grid* g, cudaError_t e, const char* where)
{
    return fail(g, PD_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define PD_CUDA(g, call)                                  \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(g, e_, #call); \
    } while (0)

bool valid_desc(const pd_grid_desc& d, std::string& why)
{
    if (d.n_xi < 2 || d.n_eta < 2) { why = "n_xi, n_eta must be >= 2"; return false; }
    if (d.periodic_xi && d.n_xi < 3) { why = "periodic xi needs n_xi >= 3"; return false; }
    if (d.m_xi < 3 || d.m_eta < 3 || d.m_xi > kMaxM || d.m_eta > kMaxM) { why = "m must be in [3, 32]"; return false; }
    if (!(d.h_ratio_xi > 0 && d.h_ratio_xi < 1 && d.h_ratio_eta > 0 && d.h_ratio_eta < 1)) {
        why = "patch ratio h / Delta must lie in (0, 1)"; return false;
    }
    if (d.k_micro < 1 || d.k_micro > kMaxK) { why = "k_micro must be in [1, 4096]"; return false; }
    if (d.micro_solver != PD_MICRO_FE && d.micro_solver != PD_MICRO_ADI) { why = "unknown micro solver"; return false; }
    if (!(d.dt_micro >= 0) || !std::isfinite(d.dt_micro)) { why = "dt_micro must be >= 0 and finite"; return false; }
    if (d.dt_micro == 0 && !(d.cfl_micro > 0 && d.cfl_micro <= 1)) { why = "cfl_micro must be in (0, 1]"; return false; }
    if (d.micro_solver == PD_MICRO_ADI && !(d.m_xi == d.m_eta && (d.m_xi == 3 || d.m_xi == 5 || d.m_xi == 7 || d.m_xi == 9 || d.m_xi == 11))) {
        why = "the ADI micro solver needs m_xi == m_eta in {3,5,7,9,11}"; return false;
    }
    if (!(d.xi1 > d.xi0) || !(d.eta1 > d.eta0)) { why = "empty computational box"; return false; }
    if (d.map < 0 || d.map > 3) { why = "unknown map"; return false; }
    if (d.prec != PD_FP32 && d.prec != PD_FP64) { why = "unknown precision"; return false; }
    if (d.conv_scheme != PD_CONV_UPWIND && d.conv_scheme != PD_CONV_CENTRAL) { why = "unknown convection scheme"; return false; }
    if (d.restrict_mode != PD_RESTRICT_LIFTED && d.restrict_mode != PD_RESTRICT_MACRO) { why = "unknown restriction"; return false; }
    if (d.map == PD_MAP_POLAR && !(d.map_p[0] > 0 && d.map_p[1] > d.map_p[0])) { why = "polar map needs 0 < r_in < r_out"; return false; }
    if (d.map == PD_MAP_SINE && !(std::fabs(d.map_p[0]) < 1)) { why = "sine stretching needs |lambda| < 1"; return false; }
    long long np = (long long)(d.periodic_xi ? d.n_xi : d.n_xi - 1) * (d.n_eta - 1);
    if (np * d.m_xi * d.m_eta > (1LL << 40)) { why = "problem too large"; return false; }
    return true;
}

// monomial coefficients of the Lagrange basis on {-D, 0, D}: ell_p(s) = sum_k L[p][k] s^k
void lagrange_monomials(double D, double L[3][3])
{
    L[0][0] = 0;   L[0][1] = -0.5 / D; L[0][2] = 0.5 / (D * D);
    L[1][0] = 1;   L[1][1] = 0;        L[1][2] = -1.0 / (D * D);
    L[2][0] = 0;   L[2][1] = 0.5 / D;  L[2][2] = 0.5 / (D * D);
}

void poly_weights(InstDev& I)
{
    double Lx[3][3], Ly[3][3];
    lagrange_monomials(I.Dx, Lx);
    lagrange_monomials(I.Dy, Ly);
    const int kl[9][2] = { {0, 0}, {1, 0}, {0, 1}, {2, 0}, {1, 1}, {0, 2}, {2, 1}, {1, 2}, {2, 2} };
    for (int r = 0; r < 9; ++r)
        for (int p = 0; p < 3; ++p)
            for (int q = 0; q < 3; ++q) I.lw[r][p * 3 + q] = Lx[p][kl[r][0]] * Ly[q][kl[r][1]];
    // row 0: C0 = c00 - h_xi^2 c20 / 12 - h_eta^2 c02 / 12 (eq. C_0)
    for (int jj = 0; jj < 9; ++jj)
        I.lw[0][jj] -= I.hx * I.hx / 12.0 * I.lw[3][jj] + I.hy * I.hy / 12.0 * I.lw[5][jj];
    // two-phase form over the differences (slot: 0 S-, 1 S0, 2 S+, 3 D-, 4 D0, 5 D+, 6 T, 7 V, 8 U00):
    // S_q = U(-1,q) - 2U(0,q) + U(1,q), D_q = U(1,q) - U(-1,q), T = U(0,1) - U(0,-1),
    // V = U(0,-1) - 2U(0,0) + U(0,1)
    const double Dx = I.Dx, Dy = I.Dy;
    const int sl[9][3] = { {8, 1, 7}, {4, 4, 4}, {6, 6, 6}, {1, 1, 1}, {5, 3, 3}, {7, 7, 7}, {2, 0, 0}, {5, 3, 4}, {2, 0, 1} };
    const double ww[9][3] = {
        { -I.hx * I.hx / (24.0 * Dx * Dx), -I.hy * I.hy / (24.0 * Dy * Dy), 1.0 },   // C0
        { 0.0, 0.0, 1.0 / (2.0 * Dx) },                                              // c10
        { 0.0, 0.0, 1.0 / (2.0 * Dy) },                                              // c01
        { 0.0, 0.0, 1.0 / (2.0 * Dx * Dx) },                                         // c20
        { -1.0, 0.0, 1.0 / (4.0 * Dx * Dy) },                                        // c11
        { 0.0, 0.0, 1.0 / (2.0 * Dy * Dy) },                                         // c02
        { -1.0, 0.0, 1.0 / (4.0 * Dx * Dx * Dy) },                                   // c21
        { 1.0, -2.0, 1.0 / (4.0 * Dx * Dy * Dy) },                                   // c12
        { 1.0, -2.0, 1.0 / (4.0 * Dx * Dx * Dy * Dy) },                              // c22
    };
    for (int k = 0; k < 9; ++k)
        for (int c = 0; c < 3; ++c) { I.c2slot[k][c] = sl[k][c]; I.c2w[k][c] = ww[k][c]; }
}

void fill_inst(Inst& s, long long u_off, long long p_off, long long pt_off, long long e_off)
{
    const pd_grid_desc& d = s.d;
    InstDev& I = s.I;
    std::memset(&I, 0, sizeof(I));
    I.n_xi = d.n_xi; I.n_eta = d.n_eta; I.periodic = d.periodic_xi ? 1 : 0;
    I.nxp = I.periodic ? d.n_xi : d.n_xi + 1;
    I.nyp = d.n_eta + 1;
    I.ncols = I.periodic ? d.n_xi : d.n_xi - 1;
    I.nrows = d.n_eta - 1;
    I.i0 = I.periodic ? 0 : 1;
    I.mx = d.m_xi; I.my = d.m_eta; I.K = d.k_micro;
    I.conv = d.conv_scheme; I.restrict_mode = d.restrict_mode; I.map = d.map;
    I.micro = d.micro_solver;
    I.n_patch = I.ncols * I.nrows;
    I.xi0 = d.xi0; I.xi1 = d.xi1; I.eta0 = d.eta0; I.eta1 = d.eta1;
    I.Dx = (d.xi1 - d.xi0) / d.n_xi;
    I.Dy = (d.eta1 - d.eta0) / d.n_eta;
    I.hx = d.h_ratio_xi * I.Dx;
    I.hy = d.h_ratio_eta * I.Dy;
    I.dx = I.hx / (d.m_xi - 1);
    I.dy = I.hy / (d.m_eta - 1);
    for (int k = 0; k < 4; ++k) I.map_p[k] = d.map_p[k];
    I.u_off = u_off; I.p_off = p_off; I.pt_off = pt_off; I.e_off = e_off;
    I.inv_dx = 1.0 / I.dx; I.inv_dy = 1.0 / I.dy;
    I.inv_dx2 = 1.0 / (I.dx * I.dx); I.inv_dy2 = 1.0 / (I.dy * I.dy);
    I.inv_4dxdy = 1.0 / (4.0 * I.dx * I.dy);
    I.ppw = 32 / d.m_xi;
    I.coef_mode = COEF_RECORDS;
    I.edge_stride = (d.m_xi > d.m_eta ? d.m_xi : d.m_eta) + 2;
    poly_weights(I);
    s.bnd_host.clear();
    for (int j = 0; j < I.nyp; ++j)
        for (int i = 0; i < I.nxp; ++i) {
            bool b = (j == 0 || j == I.nyp - 1) || (!I.periodic && (i == 0 || i == I.nxp - 1));
            if (b) s.bnd_host.push_back(make_int2(i, j));
        }
    I.n_bnd = (int)s.bnd_host.size();
}

// Z_k(mu r) = J_k(mu ra) Y_k(mu r) - Y_k(mu ra) J_k(mu r); first root of Z_k(mu rb)
double bessel_cross(int k, double mu, double ra, double r)
{
    return std::cyl_bessel_j((double)k, mu * ra) * std::cyl_neumann((double)k, mu * r)
         - std::cyl_neumann((double)k, mu * ra) * std::cyl_bessel_j((double)k, mu * r);
}

double first_root(int k, double ra, double rb)
{
    double h = 0.02 * M_PI / (rb - ra);
    double lo = h, flo = bessel_cross(k, lo, ra, rb);
    for (int it = 0; it < 200000; ++it) {
        double hi = lo + h, fhi = bessel_cross(k, hi, ra, rb);
        if ((flo < 0) != (fhi < 0)) {
            for (int b = 0; b < 200 && hi - lo > 1e-15 * hi; ++b) {
                double mid = 0.5 * (lo + hi), fm = bessel_cross(k, mid, ra, rb);
                if ((fm < 0) == (flo < 0)) { lo = mid; flo = fm; } else hi = mid;
            }
            return 0.5 * (lo + hi);
        }
        lo = hi; flo = fhi;
    }
    return NAN;
}

pd_status check_inst(pd_grid* g, int inst)
{
    if (!g) return PD_EINVAL;
    if (inst < 0 || inst >= (int)g->inst.size()) return fail(g, PD_EINVAL, "instance index out of range");
    return PD_OK;
}

pd_status all_coeffs_set(pd_grid* g)
{
    for (size_t k = 0; k < g->inst.size(); ++k)
        if (!g->inst[k].coef_set) return fail(g, PD_ESTATE, "pd_set_coeffs not called for instance " + std::to_string(k));
    return PD_OK;
}

// micro-state layout over all instances: section of each kind holds every
// instance's patches back to back (per-instance offsets pt_off / e_off / p_off)
void layout(const pd_grid* g, const Inst& s, pd_info& o)
{
    long long pts = 0, edges = 0;
    bool fp32 = s.d.prec == PD_FP32;
    for (auto& t : g->inst) {
        pts += (long long)t.I.n_patch * t.I.mx * t.I.my;
        edges += (long long)t.I.n_patch * 4 * t.I.edge_stride;
    }
    size_t es = fp32 ? 4 : 8;
    o.edge_stride = s.I.edge_stride;
    o.off_u0 = align256(kStateHeader);
    o.off_r = align256(o.off_u0 + (size_t)pts * 8);
    o.off_w = align256(o.off_r + (size_t)pts * es);
    o.off_edge = align256(o.off_w + (size_t)pts * es);
    o.off_bias = align256(o.off_edge + (size_t)edges * 8);
    o.state_bytes = align256(o.off_bias + (size_t)g->n_patch_total * 8);
}

pd_status ensure_step_buffers(pd_grid* g, int n_macro)
{
    size_t nf = 0;
    for (auto& s : g->inst) nf = std::max(nf, (size_t)s.n_item);
    if (nf > g->flags_n) {
        if (g->flags) { cudaStreamSynchronize(g->stream); cudaFree(g->flags); }
        PD_CUDA(g, cudaMalloc(&g->flags, sizeof(int) * nf));
        g->flags_n = nf;
    }
    if (!g->U_scratch) {
        PD_CUDA(g, cudaMalloc(&g->U_scratch, sizeof(double) * g->n_macro_total));
        g->U_scratch_n = (size_t)g->n_macro_total;
    }
    size_t need = 0;
    for (auto& s : g->inst) need += (size_t)n_macro * (s.d.k_micro + kTabExtra);
    if (need > g->tab_n) {
        if (g->tab) {
            cudaStreamSynchronize(g->stream);
            cudaFree(g->tab);
            for (auto& kv : g->gcache) { cudaGraphExecDestroy(kv.second.exec); cudaGraphDestroy(kv.second.graph); }
            g->gcache.clear();
        }
        PD_CUDA(g, cudaMalloc(&g->tab, sizeof(double) * need));
        g->tab_n = need;
    }
    return PD_OK;
}

// sequence of kernels for n_macro steps on stream st (captured or direct)
pd_status enqueue_steps(pd_grid* g, double* U, int n_macro, const std::vector<double>& dtm, cudaStream_t st, int& n_launch)
{
    size_t tab_off = 0;
    for (size_t k = 0; k < g->inst.size(); ++k) {
        Inst& s = g->inst[k];
        const InstDev& I = s.I;
        double* bufs[2] = { U + I.u_off, g->U_scratch + I.u_off };
        int stride = I.K + kTabExtra;
        if (g->persist && I.micro == PD_MICRO_FE && persist_fits(I, s.d.prec)) {
            int chunk = persist_max_steps(I, s.d.prec);
            for (int s0 = 0; s0 < n_macro; s0 += chunk) {
                PersistArgs pa;
                pa.U0 = bufs[0]; pa.U1 = bufs[1];
                pa.tab = g->tab + tab_off;
                pa.s0 = s0; pa.n_steps = std::min(chunk, n_macro - s0);
                pa.dtm = dtm[k];
                pa.flags = g->flags;
                pa.bnd_off = s.bnd_off; pa.bnd_idx = s.bnd_idx;
                pa.wait_ns = g->wait_ns;
                pa.silent_warp = g->silent_warp;
                cudaError_t e = cudaMemsetAsync(g->flags, 0, sizeof(int) * s.n_item, st);
                if (e == cudaSuccess) e = launch_persist(I, s.d.prec, pa, st);
                if (e != cudaSuccess) return cuda_fail(g, e, "persistent step");
                n_launch += 1;
            }
            if (n_macro & 1) {
                cudaError_t e = cudaMemcpyAsync(bufs[0], bufs[1], sizeof(double) * (size_t)I.nxp * I.nyp,
                                                cudaMemcpyDeviceToDevice, st);
                if (e != cudaSuccess) return cuda_fail(g, e, "copy back");
            }
        } else if (fused_supported(I)) {
            for (int t = 0; t < n_macro; ++t) {
                cudaError_t e = launch_fused_step(I, nullptr, s.d.prec, bufs[t & 1], bufs[(t + 1) & 1],
                                                  g->tab + tab_off + (size_t)t * stride, dtm[k], st, &n_launch);
                if (e != cudaSuccess) return cuda_fail(g, e, "fused step");
            }
            if (n_macro & 1) {
                cudaError_t e = cudaMemcpyAsync(bufs[0], bufs[1], sizeof(double) * (size_t)I.nxp * I.nyp,
                                                cudaMemcpyDeviceToDevice, st);
                if (e != cudaSuccess) return cuda_fail(g, e, "copy back");
            }
        } else {
            return fail(g, PD_EINVAL, "fused step needs m_xi == m_eta in {3,5,7,9,11}");
        }
        tab_off += (size_t)n_macro * stride;
    }
    return PD_OK;
}

// pd_step with a second-order outer integrator: one instance, fused kernels
pd_status step_higher(pd_grid* g, double* U, double t0, double dtm, int n_macro)
{
    Inst& s = g->inst[0];
    const InstDev& I = s.I;
    pd_status rc = ensure_step_buffers(g, n_macro + 1);
    if (rc) return rc;
    const size_t nf = (size_t)g->n_macro_total;
    if (!g->S2) PD_CUDA(g, cudaMalloc(&g->S2, sizeof(double) * nf));
    if (!g->dUa) {
        PD_CUDA(g, cudaMalloc(&g->dUa, sizeof(double) * (size_t)g->n_patch_total));
        PD_CUDA(g, cudaMalloc(&g->dUb, sizeof(double) * (size_t)g->n_patch_total));
    }
    cudaStream_t st = g->stream;
    const int stride = I.K + kTabExtra;
    PD_CUDA(g, launch_time_table(I, t0, dtm, n_macro + 1, g->tab, st));
    int nl = 1;
    auto row = [&](int k) { return g->tab + (size_t)k * stride; };
    auto heun = [&](int k) -> pd_status {
        cudaError_t e = launch_fused_step(I, nullptr, s.d.prec, U, g->U_scratch, row(k), dtm, st, &nl);
        if (e == cudaSuccess) e = launch_fused_step(I, nullptr, s.d.prec, g->U_scratch, g->S2, row(k + 1), dtm, st, &nl);
        if (e == cudaSuccess) { e = launch_heun_combine(I, U, g->U_scratch, g->S2, st); ++nl; }
        if (e != cudaSuccess) return cuda_fail(g, e, "Heun step");
        return PD_OK;
    };
    if (g->integrator == PD_INT_HEUN) {
        for (int k = 0; k < n_macro && !rc; ++k) rc = heun(k);
    } else {
        // AB2: the history starts with the restricted change at T_0, the first step is Heun's
        double* cur = g->dUb;
        double* prev = g->dUa;
        cudaError_t e = launch_patch_dU(I, s.d.prec, U, row(0), I.K, prev, nullptr, nullptr, st);
        ++nl;
        if (e != cudaSuccess) return cuda_fail(g, e, "AB2 history");
        rc = heun(0);
        for (int k = 1; k < n_macro && !rc; ++k) {
            e = launch_patch_dU(I, s.d.prec, U, row(k), I.K, cur, nullptr, nullptr, st);
            if (e == cudaSuccess) e = launch_ab2(I, U, cur, prev, t0 + k * dtm, dtm, st);
            nl += 2;
            if (e != cudaSuccess) return cuda_fail(g, e, "AB2 step");
            std::swap(cur, prev);
        }
    }
    g->launches += nl;
    return rc;
}

// pd_step with the edge data refreshed q times per burst, through the separate
// passes: lift; q bursts of K/q steps, each but the first preceded by a
// restriction (restricted change so far) and a refresh of the edge forcing;
// restriction of the whole burst; projection
pd_status step_refresh(pd_grid* g, double* U, double t0, const std::vector<double>& dtm, int n_macro)
{
    if (!g->state) {
        PD_CUDA(g, cudaMalloc(&g->state, g->state_bytes));
        PD_CUDA(g, cudaMalloc(&g->dU, sizeof(double) * g->n_patch_total));
    }
    if (!g->Dq) {
        PD_CUDA(g, cudaMalloc(&g->Dq, sizeof(double) * (size_t)g->n_macro_total));
        PD_CUDA(g, cudaMalloc(&g->dRa, sizeof(double) * (size_t)g->n_patch_total));
        PD_CUDA(g, cudaMalloc(&g->dRb, sizeof(double) * (size_t)g->n_patch_total));
        PD_CUDA(g, cudaMalloc(&g->dRz, sizeof(double) * (size_t)g->n_patch_total));
        PD_CUDA(g, cudaMemsetAsync(g->dRz, 0, sizeof(double) * (size_t)g->n_patch_total, g->stream));
    }
    const int Q = g->q_refresh;
    for (int t = 0; t < n_macro; ++t) {
        for (size_t k = 0; k < g->inst.size(); ++k) {
            Inst& s = g->inst[k];
            const InstDev& I = s.I;
            pd_info lay;
            layout(g, s, lay);
            const double T = t0 + t * dtm[k];
            const int Ks = I.K / Q;
            // restricted changes of the departure alone (no reference bias, whose
            // subtraction would cancel digits); zero before the first sub-burst
            double* cur = g->dRa;
            const double* prev = g->dRz;
            cudaError_t e = launch_lift(I, nullptr, s.d.prec, U + I.u_off, T, g->state, lay, g->stream);
            for (int q = 0; q < Q && e == cudaSuccess; ++q) {
                const double Tq = T + q * Ks * I.dt;
                if (q > 0) {
                    e = launch_restrict(I, s.d.prec, g->state, lay, cur, g->stream, g->dRz);
                    if (e == cudaSuccess)
                        e = launch_refresh(I, s.d.prec, U + I.u_off, cur, prev, T + (q - 1) * Ks * I.dt, Tq, q == 1,
                                           g->Dq + I.u_off, g->state + lay.off_r, g->stream);
                    prev = cur;
                    cur = (cur == g->dRa) ? g->dRb : g->dRa;
                    g->launches += 3;
                }
                if (e == cudaSuccess) e = launch_burst(I, nullptr, s.d.prec, g->state, lay, Tq, Ks, g->stream);
                g->launches += 2;
            }
            if (e == cudaSuccess) e = launch_restrict(I, s.d.prec, g->state, lay, g->dU, g->stream);
            if (e == cudaSuccess) e = launch_project(I, U + I.u_off, g->dU, T, dtm[k], g->stream);
            if (e != cudaSuccess) return cuda_fail(g, e, "step with edge refresh");
            g->launches += 4;
        }
    }
    return PD_OK;
}

pd_status step_fallback(pd_grid* g, double* U, double t0, const std::vector<double>& dtm, int n_macro)
{
    // separate passes through an internal state buffer (m not covered by the fused kernel)
    if (!g->state) {
        PD_CUDA(g, cudaMalloc(&g->state, g->state_bytes));
        PD_CUDA(g, cudaMalloc(&g->dU, sizeof(double) * g->n_patch_total));
    }
    for (int t = 0; t < n_macro; ++t) {
        for (size_t k = 0; k < g->inst.size(); ++k) {
            Inst& s = g->inst[k];
            pd_info lay;
            layout(g, s, lay);
            double T = t0 + t * dtm[k];
            cudaError_t e = launch_lift(s.I, nullptr, s.d.prec, U + s.I.u_off, T, g->state, lay, g->stream);
            if (e == cudaSuccess) e = launch_burst(s.I, nullptr, s.d.prec, g->state, lay, T, s.I.K, g->stream);
            if (e == cudaSuccess) e = launch_restrict(s.I, s.d.prec, g->state, lay, g->dU, g->stream);
            if (e == cudaSuccess) e = launch_project(s.I, U + s.I.u_off, g->dU, T, dtm[k], g->stream);
            if (e != cudaSuccess) return cuda_fail(g, e, "step (separate passes)");
            g->launches += 6;
        }
    }
    return PD_OK;
}


// ---------------------------------------------------------------------------
// batched execution

bool use_batch(const pd_grid* g)
{
    if (g->inst.size() > 1) return true;
    for (auto& s : g->inst) if (s.I.coef_mode != COEF_RECORDS) return true;
    return false;
}

bool all_batch_supported(const pd_grid* g)
{
    for (auto& s : g->inst) if (!batch_supported(s.I)) return false;
    return true;
}

pd_status prepare_batch(pd_grid* g)
{
    if (!g->batch_dirty) return PD_OK;
    PD_CUDA(g, cudaStreamSynchronize(g->stream));   // no kernel may still read the old tables
    g->dtm_host.clear();                            // tau may have changed: rebuild the update scales
    size_t n = g->inst.size();
    std::vector<InstDev> host(n);
    std::vector<BatchItem> items;
    for (size_t k = 0; k < n; ++k) {
        Inst& s = g->inst[k];
        int P = 32 / s.I.mx;
        s.I.ppw = g->bt_half ? std::max(1, (P + 1) / 2) : P;
        host[k] = s.I;
    }
    // per micro size (largest first): on FP32 grids one class of the separable-map
    // instances' patch groups, then one of the other instances' patch groups and
    // every instance's boundary chunks (either may be empty and is then skipped)
    std::vector<int> sizes;
    for (size_t k = 0; k < n; ++k)
        if (std::find(sizes.begin(), sizes.end(), g->inst[k].I.mx) == sizes.end()) sizes.push_back(g->inst[k].I.mx);
    std::sort(sizes.rbegin(), sizes.rend());
    g->cls_m.clear(); g->cls_beg.clear(); g->cls_n.clear(); g->cls_sep.clear();
    const bool fp32 = g->inst[0].d.prec == PD_FP32;
    auto sep_of = [&](const InstDev& I) { return fp32 && I.coef_mode == COEF_SEPARABLE; };
    for (int m : sizes) {
        for (int pass = 0; pass < 2; ++pass) {
            const bool sep = pass == 0;
            if (sep && !fp32) continue;
            const int beg = (int)items.size();
            for (size_t k = 0; k < n; ++k) {
                const InstDev& I = g->inst[k].I;
                if (I.mx != m || sep_of(I) != sep) continue;
                int wpr = (I.ncols + I.ppw - 1) / I.ppw;
                for (int jr = 0; jr < I.nrows; ++jr)
                    for (int wc = 0; wc < wpr; ++wc) items.push_back(BatchItem{ (int)k, 0, jr, wc });
            }
            if (!sep) {
                for (size_t k = 0; k < n; ++k) {
                    if (g->inst[k].I.mx != m) continue;
                    int chunks = (g->inst[k].I.n_bnd + 31) / 32;
                    for (int c = 0; c < chunks; ++c) items.push_back(BatchItem{ (int)k, 1, c, 0 });
                }
            }
            if ((int)items.size() == beg) continue;
            g->cls_m.push_back(m);
            g->cls_sep.push_back(sep ? 1 : 0);
            g->cls_beg.push_back(beg);
            g->cls_n.push_back((int)items.size() - beg);
        }
    }
    if (!g->insts_dev) PD_CUDA(g, cudaMalloc(&g->insts_dev, sizeof(InstDev) * n));
    PD_CUDA(g, cudaMemcpy(g->insts_dev, host.data(), sizeof(InstDev) * n, cudaMemcpyHostToDevice));
    cudaFree(g->items_dev);
    PD_CUDA(g, cudaMalloc(&g->items_dev, sizeof(BatchItem) * std::max<size_t>(items.size(), 1)));
    PD_CUDA(g, cudaMemcpy(g->items_dev, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice));
    g->n_items = (int)items.size();
    g->batch_dirty = false;
    for (auto& kv : g->gcache) { cudaGraphExecDestroy(kv.second.exec); cudaGraphDestroy(kv.second.graph); }
    g->gcache.clear();
    return PD_OK;
}

bool batch_needs_tables(const pd_grid* g)
{
    for (auto& s : g->inst) if (s.I.has_tsrc || s.I.sol != PD_SOL_NONE) return true;
    return false;
}

bool batch_tsrc(const pd_grid* g)
{
    for (auto& s : g->inst) if (s.I.has_tsrc) return true;
    return false;
}

pd_status batch_buffers(pd_grid* g, int n_macro, const std::vector<double>& dtm)
{
    size_t n = g->inst.size();
    if (!g->dtm_dev) PD_CUDA(g, cudaMalloc(&g->dtm_dev, sizeof(double) * n));
    if (!g->scale_dev) PD_CUDA(g, cudaMalloc(&g->scale_dev, sizeof(double2) * n));
    if (g->dtm_host != dtm) {
        std::vector<double2> sc(n);
        for (size_t k = 0; k < n; ++k) {
            const double bs = dtm[k] * g->inst[k].I.inv_tau;
            sc[k] = make_double2(bs * g->inst[k].I.inv_nn, bs);
        }
        PD_CUDA(g, cudaStreamSynchronize(g->stream));
        PD_CUDA(g, cudaMemcpy(g->dtm_dev, dtm.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
        PD_CUDA(g, cudaMemcpy(g->scale_dev, sc.data(), sizeof(double2) * n, cudaMemcpyHostToDevice));
        g->dtm_host = dtm;
    }
    // one work-queue counter per macro step and class (at most two classes for
    // each of the five batched micro sizes, so the classes may be rebuilt afterwards)
    const size_t n_counters = (size_t)n_macro * 10;
    if (n_counters > g->counters_n) {
        if (g->counters) { cudaStreamSynchronize(g->stream); cudaFree(g->counters); }
        PD_CUDA(g, cudaMalloc(&g->counters, sizeof(int) * n_counters));
        g->counters_n = n_counters;
        for (auto& kv : g->gcache) { cudaGraphExecDestroy(kv.second.exec); cudaGraphDestroy(kv.second.graph); }
        g->gcache.clear();
    }
    if (!g->U_scratch) {
        PD_CUDA(g, cudaMalloc(&g->U_scratch, sizeof(double) * g->n_macro_total));
        g->U_scratch_n = (size_t)g->n_macro_total;
    }
    return PD_OK;
}

// time tables of every instance for n_macro steps (only when some instance has a
// time-dependent source or Dirichlet data)
pd_status batch_time_tables(pd_grid* g, double t0, int n_macro, const std::vector<double>& dtm)
{
    size_t n = g->inst.size();
    std::vector<long long> off(n + 1, 0);
    for (size_t k = 0; k < n; ++k) off[k + 1] = off[k] + (long long)n_macro * (g->inst[k].I.K + kTabExtra);
    size_t need = (size_t)off[n];
    if (need > g->tab_n) {
        if (g->tab) { cudaStreamSynchronize(g->stream); cudaFree(g->tab); }
        PD_CUDA(g, cudaMalloc(&g->tab, sizeof(double) * need));
        g->tab_n = need;
        for (auto& kv : g->gcache) { cudaGraphExecDestroy(kv.second.exec); cudaGraphDestroy(kv.second.graph); }
        g->gcache.clear();
    }
    if (!g->tab_off_dev) PD_CUDA(g, cudaMalloc(&g->tab_off_dev, sizeof(long long) * (n + 1)));
    PD_CUDA(g, cudaStreamSynchronize(g->stream));
    PD_CUDA(g, cudaMemcpy(g->tab_off_dev, off.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice));
    PD_CUDA(g, launch_batch_time_tables(g->insts_dev, (int)n, g->dtm_dev, t0, n_macro, g->tab_off_dev, g->tab, off[n], g->stream));
    g->launches += 1;
    return PD_OK;
}

int batch_grid(const pd_grid* g, int block, int M, bool sep)
{
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, g->device);
    int per = batch_blocks_per_sm(g->inst[0].d.prec, batch_tsrc(g), M, sep, block);
    return std::max(1, per) * nsm;
}

// n_macro macro steps; every step launches one kernel per micro-size class
// (each sized to fill the device, its warps pulling that class's items)
pd_status enqueue_batch(pd_grid* g, double* U, int n_macro, cudaStream_t st, int& n_launch, bool tables)
{
    const int ncls = (int)g->cls_m.size();
    PD_CUDA(g, cudaMemsetAsync(g->counters, 0, sizeof(int) * (size_t)n_macro * ncls, st));
    int block = g->bt_block;
    std::vector<int> grid(ncls);
    for (int c = 0; c < ncls; ++c) grid[c] = batch_grid(g, block, g->cls_m[c], g->cls_sep[c] != 0);
    for (int t = 0; t < n_macro; ++t) {
        for (int c = 0; c < ncls; ++c) {
            if (g->cls_n[c] == 0) continue;
            BatchArgs a;
            a.insts = g->insts_dev; a.items = g->items_dev + g->cls_beg[c]; a.n_items = g->cls_n[c];
            a.counter = g->counters + (size_t)t * ncls + c;
            a.Ubase = U; a.Sbase = g->U_scratch; a.parity = t & 1;
            a.dtm = g->dtm_dev;
            a.scale = g->scale_dev;
            a.tab = tables ? g->tab : nullptr;
            a.tab_off = tables ? g->tab_off_dev : nullptr;
            a.step = t;
            cudaError_t e = launch_batch(g->inst[0].d.prec, batch_tsrc(g), g->cls_m[c], g->cls_sep[c] != 0, a, block,
                                         grid[c], st);
            if (e != cudaSuccess) return cuda_fail(g, e, "batched step");
            n_launch += 1;
        }
    }
    if (n_macro & 1) {
        cudaError_t e = cudaMemcpyAsync(U, g->U_scratch, sizeof(double) * g->n_macro_total, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_fail(g, e, "copy back");
    }
    return PD_OK;
}

// Autotuner: time a few macro steps of every candidate (threads per block x
// patches per warp) on scratch buffers and keep the fastest.
pd_status batch_autotune(pd_grid* g, int n_trial)
{
    std::vector<double> dtm(g->inst.size());
    for (size_t k = 0; k < g->inst.size(); ++k) dtm[k] = g->inst[k].dtm_sugg;
    pd_status rc = batch_buffers(g, n_trial, dtm);
    if (rc) return rc;
    double* trial = nullptr;
    PD_CUDA(g, cudaMalloc(&trial, sizeof(double) * g->n_macro_total));
    PD_CUDA(g, cudaMemsetAsync(trial, 0, sizeof(double) * g->n_macro_total, g->stream));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 1e30;
    int best_block = g->bt_block;
    bool best_half = g->bt_half;
    g->tune_log.clear();
    const int blocks[2] = { 64, 128 };
    for (int hv = 0; hv < 2; ++hv) {
        g->bt_half = hv != 0;
        g->batch_dirty = true;
        rc = prepare_batch(g);
        if (rc) break;
        bool tables = batch_needs_tables(g);
        if (tables) { rc = batch_time_tables(g, 0.0, n_trial, dtm); if (rc) break; }
        for (int bi = 0; bi < 2; ++bi) {
            g->bt_block = blocks[bi];
            int nl = 0;
            rc = enqueue_batch(g, trial, 1, g->stream, nl, tables);   // warm-up
            if (rc) break;
            cudaEventRecord(e0, g->stream);
            rc = enqueue_batch(g, trial, n_trial, g->stream, nl, tables);
            if (rc) break;
            cudaEventRecord(e1, g->stream);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            double per = ms / n_trial;
            g->tune_log.push_back(per);
            if (per < best) { best = per; best_block = blocks[bi]; best_half = g->bt_half; }
        }
        if (rc) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(g->stream);
    cudaFree(trial);
    int herr = 0;
    cudaMemcpy(&herr, g->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (herr) cudaMemset(g->err, 0, sizeof(int));   // trial runs on zero fields; nothing to report
    g->bt_block = best_block;
    g->bt_half = best_half;
    g->batch_dirty = true;
    g->bt_tuned = true;
    if (rc) return rc;
    return prepare_batch(g);
}

pd_status step_batch(pd_grid* g, double* U, double t0, const std::vector<double>& dtm, int n_macro)
{
    if (g->autotune && !g->bt_tuned) {
        pd_status rc = batch_autotune(g, 2);
        if (rc) return rc;
    }
    pd_status rc = prepare_batch(g);
    if (rc) return rc;
    rc = batch_buffers(g, n_macro, dtm);
    if (rc) return rc;
    bool tables = batch_needs_tables(g);
    if (tables) { rc = batch_time_tables(g, t0, n_macro, dtm); if (rc) return rc; }
    if (!g->graphs) {
        int nl = 0;
        rc = enqueue_batch(g, U, n_macro, g->stream, nl, tables);
        g->launches += nl;
        return rc;
    }
    GraphKey key{ (uintptr_t)U, n_macro, dtm };
    auto it = g->gcache.find(key);
    if (it == g->gcache.end()) {
        GraphEntry ge;
        PD_CUDA(g, cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal));
        int nl = 0;
        rc = enqueue_batch(g, U, n_macro, g->cap, nl, tables);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(g->cap, &graph);
        if (rc) { if (graph) cudaGraphDestroy(graph); return rc; }
        if (e != cudaSuccess) return cuda_fail(g, e, "end capture");
        e = cudaGraphInstantiate(&ge.exec, graph, 0);
        if (e != cudaSuccess) { cudaGraphDestroy(graph); return cuda_fail(g, e, "graph instantiate"); }
        ge.graph = graph;
        ge.n_nodes = nl;
        it = g->gcache.emplace(key, ge).first;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (g->timing) {
        for (cudaEvent_t* e : { &e0, &e1 }) {
            if (!g->tfree.empty()) { *e = g->tfree.back(); g->tfree.pop_back(); }
            else PD_CUDA(g, cudaEventCreate(e));
        }
        PD_CUDA(g, cudaEventRecord(e0, g->stream));
    }
    PD_CUDA(g, cudaGraphLaunch(it->second.exec, g->stream));
    g->launches += it->second.n_nodes;
    if (g->timing) {
        PD_CUDA(g, cudaEventRecord(e1, g->stream));
        g->tev.emplace_back(e0, e1);
        g->t_launches += n_macro;
    }
    return PD_OK;
}

}  // namespace

extern "C" {

int pd_abi_version(void) { return PD_ABI_VERSION; }

const char* pd_status_str(pd_status s)
{
    switch (s) {
    case PD_OK: return "ok";
    case PD_EINVAL: return "invalid argument";
    case PD_ENOMEM: return "out of device memory";
    case PD_ECUDA: return "CUDA error";
    case PD_ESTATE: return "call out of order";
    case PD_EUNSTABLE: return "step above the stability bound";
    case PD_ETIMEOUT: return "device wait timed out";
    case PD_ENUMERIC: return "non-finite values on the device";
    }
    return "unknown status";
}

const char* pd_last_error(const pd_grid* g) { return g ? g->last.c_str() : "null grid"; }

long long pd_launch_count(const pd_grid* g) { return g ? g->launches : 0; }

pd_status pd_create_grid(const pd_grid_desc* descs, int n_inst, void* cuda_stream, pd_grid** out)
{
    NvtxRange nvtx_range("pd_create_grid");
    if (!descs || n_inst < 1 || !out) return PD_EINVAL;
    *out = nullptr;
    pd_grid* g = new pd_grid();
    g->stream = (cudaStream_t)cuda_stream;
    cudaGetDevice(&g->device);
    long long u_off = 0, p_off = 0, pt_off = 0, e_off = 0;
    g->inst.resize(n_inst);
    for (int k = 0; k < n_inst; ++k) {
        std::string why;
        if (!valid_desc(descs[k], why)) {
            delete g;
            return PD_EINVAL;
        }
        if (k > 0 && descs[k].prec != descs[0].prec) {
            delete g;
            return PD_EINVAL;
        }
        if (n_inst > 1 && descs[k].micro_solver != PD_MICRO_FE) {   // ADI runs on one-instance grids
            delete g;
            return PD_EINVAL;
        }
        g->inst[k].d = descs[k];
        fill_inst(g->inst[k], u_off, p_off, pt_off, e_off);
        u_off += (long long)g->inst[k].I.nxp * g->inst[k].I.nyp;
        p_off += g->inst[k].I.n_patch;
        pt_off += (long long)g->inst[k].I.n_patch * g->inst[k].I.mx * g->inst[k].I.my;
        e_off += (long long)g->inst[k].I.n_patch * 4 * g->inst[k].I.edge_stride;
    }
    g->n_macro_total = u_off;
    g->n_patch_total = p_off;
    cudaError_t e = cudaMalloc(&g->err, sizeof(int) * 4);
    if (e == cudaSuccess) e = cudaMemset(g->err, 0, sizeof(int) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&g->acc, sizeof(unsigned long long) * 4);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking);
    for (int k = 0; k < n_inst && e == cudaSuccess; ++k) {
        Inst& s = g->inst[k];
        e = cudaMalloc(&s.bnd_ij, sizeof(int2) * (s.I.n_bnd + 1));
        if (e == cudaSuccess) e = cudaMalloc(&s.bnd_xy, sizeof(double2) * (s.I.n_bnd + 1));
        if (e == cudaSuccess && s.I.n_bnd)
            e = cudaMemcpy(s.bnd_ij, s.bnd_host.data(), sizeof(int2) * s.I.n_bnd, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) {
            // owner item warp of every boundary node: the warp of the nearest patch
            int P = 32 / s.I.mx;
            int wpr = (s.I.ncols + P - 1) / P;
            s.n_item = wpr * s.I.nrows;
            std::vector<std::vector<int>> own(s.n_item);
            for (int k = 0; k < s.I.n_bnd; ++k) {
                int ii = s.bnd_host[k].x, jj = s.bnd_host[k].y;
                int ic = std::min(std::max(ii - s.I.i0, 0), s.I.ncols - 1);
                int jr = std::min(std::max(jj - 1, 0), s.I.nrows - 1);
                own[jr * wpr + ic / P].push_back(k);
            }
            std::vector<int> off(s.n_item + 1, 0), idx;
            for (int w = 0; w < s.n_item; ++w) {
                off[w + 1] = off[w] + (int)own[w].size();
                idx.insert(idx.end(), own[w].begin(), own[w].end());
            }
            idx.push_back(0);
            e = cudaMalloc(&s.bnd_off, sizeof(int) * off.size());
            if (e == cudaSuccess) e = cudaMalloc(&s.bnd_idx, sizeof(int) * idx.size());
            if (e == cudaSuccess) e = cudaMemcpy(s.bnd_off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMemcpy(s.bnd_idx, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice);
        }
        s.I.rec = s.rec; s.I.brec = s.brec; s.I.bnd_ij = s.bnd_ij; s.I.bnd_xy = s.bnd_xy; s.I.err = g->err;
    }
    if (e != cudaSuccess) {
        pd_destroy_grid(g);
        return e == cudaErrorMemoryAllocation ? PD_ENOMEM : PD_ECUDA;
    }
    pd_info lay;
    layout(g, g->inst[0], lay);
    g->state_bytes = lay.state_bytes;
    *out = g;
    return PD_OK;
}

pd_status pd_destroy_grid(pd_grid* g)
{
    NvtxRange nvtx_range("pd_destroy_grid");
    if (!g) return PD_EINVAL;
    DeviceGuard dg(g->device);
    if (g->stream) cudaStreamSynchronize(g->stream);
    for (auto& kv : g->gcache) { cudaGraphExecDestroy(kv.second.exec); cudaGraphDestroy(kv.second.graph); }
    for (auto& pr : g->tev) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
    for (auto e : g->tfree) cudaEventDestroy(e);
    for (auto& s : g->inst) { cudaFree(s.rec); cudaFree(s.brec); cudaFree(s.arec_c); cudaFree(s.arec_r); cudaFree(s.bnd_off); cudaFree(s.bnd_idx); cudaFree(s.col_tab); cudaFree(s.row_tab); cudaFree(s.col_tab_f); cudaFree(s.row_tab_f); cudaFree(s.bnd_ij); cudaFree(s.bnd_xy); cudaFree(s.amp); }
    cudaFree(g->err); cudaFree(g->acc); cudaFree(g->U_scratch); cudaFree(g->tab);
    cudaFree(g->S2); cudaFree(g->dUa); cudaFree(g->dUb);
    cudaFree(g->Dq); cudaFree(g->dRa); cudaFree(g->dRb); cudaFree(g->dRz);
    cudaFree(g->state); cudaFree(g->dU); cudaFree(g->flags);
    cudaFree(g->insts_dev); cudaFree(g->items_dev); cudaFree(g->dtm_dev); cudaFree(g->scale_dev); cudaFree(g->tab_off_dev); cudaFree(g->counters);
    if (g->cap) cudaStreamDestroy(g->cap);
    delete g;
    return PD_OK;
}

pd_status pd_set_stream(pd_grid* g, void* st)
{
    if (!g) return PD_EINVAL;
    g->stream = (cudaStream_t)st;
    return PD_OK;
}

pd_status pd_set_graph_mode(pd_grid* g, int enabled)
{
    if (!g) return PD_EINVAL;
    g->graphs = enabled != 0;
    return PD_OK;
}

pd_status pd_set_coeffs(pd_grid* g, int inst, const pd_coeff_desc* c)
{
    NvtxRange nvtx_range("pd_set_coeffs");
    pd_status rc = check_inst(g, inst);
    if (rc) return rc;
    if (!c) return fail(g, PD_EINVAL, "null coefficient descriptor");
    if (c->src < 0 || c->src > 3 || c->tkind < 0 || c->tkind > 2 || c->sol < 0 || c->sol > 2)
        return fail(g, PD_EINVAL, "unknown source, time or solution kind");
    if (c->n_four < 0 || c->n_four > 3) return fail(g, PD_EINVAL, "n_four must be in [0, 3]");
    if (c->n_four > 0 && !(c->four_rb > c->four_ra)) return fail(g, PD_EINVAL, "four_rb must exceed four_ra");
    if (c->src == PD_SRC_GAUSS_PATCH && !c->src_amp) return fail(g, PD_EINVAL, "GAUSS_PATCH needs src_amp");
    Inst& s = g->inst[inst];
    DeviceGuard dg(g->device);
    if (c->src == PD_SRC_GAUSS_PATCH) {
        if (!s.amp) PD_CUDA(g, cudaMalloc(&s.amp, sizeof(double) * s.I.n_patch));
        PD_CUDA(g, cudaMemcpyAsync(s.amp, c->src_amp, sizeof(double) * s.I.n_patch, cudaMemcpyHostToDevice, g->stream));
    }
    s.coef = *c;
    s.coef.src_amp = nullptr;
    s.I.sol = c->sol; s.I.tkind = c->tkind; s.I.tc = c->tc;
    // coefficient storage: 1-D metric tables when K, v, f are constant and there is
    // no source (constant-coefficient instances on separable or polar maps), else
    // per-point records
    bool tabular = c->dx == 0 && c->dy == 0 && c->ds == 0 && c->n_four == 0 && c->va[1] == 0 && c->va[2] == 0
                && c->vb[1] == 0 && c->vb[2] == 0 && c->src == PD_SRC_NONE;
    bool use_tables = tabular && s.d.micro_solver == PD_MICRO_FE
                   && (g->storage == 2 || (g->storage == 0 && g->inst.size() > 1));
    size_t es = s.d.prec == PD_FP32 ? 4 : 8;
    size_t npts = (size_t)s.I.n_patch * s.I.mx * s.I.my;
    if (use_tables) {
        s.I.coef_mode = s.d.map == PD_MAP_POLAR ? COEF_POLAR : COEF_SEPARABLE;
        if (!s.col_tab) PD_CUDA(g, cudaMalloc(&s.col_tab, sizeof(double) * 2 * (size_t)s.I.ncols * s.I.mx));
        if (!s.row_tab) PD_CUDA(g, cudaMalloc(&s.row_tab, sizeof(double) * 4 * (size_t)s.I.nrows * s.I.my));
        if (!s.col_tab_f) PD_CUDA(g, cudaMalloc(&s.col_tab_f, sizeof(float) * 2 * (size_t)s.I.ncols * s.I.mx));
        if (!s.row_tab_f) PD_CUDA(g, cudaMalloc(&s.row_tab_f, sizeof(float) * 4 * (size_t)s.I.nrows * s.I.my));
        s.I.col_tab = s.col_tab; s.I.row_tab = s.row_tab;
        s.I.col_tab_f = s.col_tab_f; s.I.row_tab_f = s.row_tab_f;
        s.I.K11 = c->d0 * c->M11; s.I.K12 = c->d0 * c->M12; s.I.K22 = c->d0 * c->M22;
        s.I.v1 = c->va[0]; s.I.v2 = c->vb[0]; s.I.f0 = c->f0;
        cudaFree(s.rec); cudaFree(s.brec); cudaFree(s.arec_c); cudaFree(s.arec_r);
        s.rec = s.brec = s.arec_c = s.arec_r = nullptr;
    } else {
        s.I.coef_mode = COEF_RECORDS;
        if (!s.rec) {
            cudaError_t ea = cudaMalloc(&s.rec, npts * 8 * es);
            if (ea == cudaSuccess) ea = cudaMalloc(&s.brec, npts * 16 * es);
            if (ea != cudaSuccess) return fail(g, ea == cudaErrorMemoryAllocation ? PD_ENOMEM : PD_ECUDA, "coefficient records");
        }
        if (s.d.micro_solver == PD_MICRO_ADI && !s.arec_c) {
            cudaError_t ea = cudaMalloc(&s.arec_c, npts * 8 * es);
            if (ea == cudaSuccess) ea = cudaMalloc(&s.arec_r, npts * 8 * es);
            if (ea != cudaSuccess) return fail(g, ea == cudaErrorMemoryAllocation ? PD_ENOMEM : PD_ECUDA, "ADI records");
        }
    }
    s.I.rec = s.rec; s.I.brec = s.brec; s.I.arec_c = s.arec_c; s.I.arec_r = s.arec_r;
    g->batch_dirty = true;
    s.I.has_tsrc = (c->src != PD_SRC_NONE && c->tkind != PD_TIME_CONST) ? 1 : 0;
    PD_CUDA(g, cudaMemsetAsync(g->acc, 0, sizeof(unsigned long long) * 4, g->stream));
    PD_CUDA(g, cudaMemsetAsync(g->err, 0, sizeof(int) * 4, g->stream));
    PD_CUDA(g, launch_precompute(s.I, *c, s.amp, s.rec, s.d.prec, g->acc, g->acc + 1, g->stream));
    g->launches += 3;
    if (use_tables) {
        PD_CUDA(g, launch_tables(s.I, s.col_tab, s.row_tab, s.col_tab_f, s.row_tab_f, nullptr, nullptr, g->stream));
        g->launches += 1;
    }
    unsigned long long h[2];
    int herr = 0;
    PD_CUDA(g, cudaMemcpyAsync(h, g->acc, sizeof(h), cudaMemcpyDeviceToHost, g->stream));
    PD_CUDA(g, cudaMemcpyAsync(&herr, g->err, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
    PD_CUDA(g, cudaStreamSynchronize(g->stream));
    if (herr & ERR_JACOBIAN) return fail(g, PD_EINVAL, "singular mapping or non-finite coefficients");
    double rate, mrate;
    std::memcpy(&rate, &h[0], sizeof(double));
    std::memcpy(&mrate, &h[1], sizeof(double));
    if (!(rate > 0)) return fail(g, PD_EINVAL, "zero operator: no micro step bound");
    if (s.d.dt_micro > 0) {
        // fixed micro step; forward Euler must stay within its explicit bound
        if (s.d.micro_solver == PD_MICRO_FE && s.d.dt_micro * rate > 1.0)
            return fail(g, PD_EUNSTABLE, "dt_micro above the explicit forward-Euler bound");
        s.dt = s.d.dt_micro;
    } else {
        s.dt = s.d.cfl_micro / rate;
    }
    s.tau = s.d.k_micro * s.dt;
    s.dtm_sugg = mrate > 0 ? 0.5 / mrate : s.tau;
    s.I.dt = s.dt; s.I.tau = s.tau;
    fill_float_consts(s.I);
    s.I.inv_tau = 1.0 / s.tau;
    s.I.inv_nn = 1.0 / ((double)(s.d.m_xi - 1) * (s.d.m_eta - 1));
    if (!use_tables) {
        PD_CUDA(g, launch_burst_records(s.I, s.d.prec, s.brec, g->stream));
        g->launches += 1;
        if (s.d.micro_solver == PD_MICRO_ADI) {
            PD_CUDA(g, launch_adi_records(s.I, s.d.prec, s.arec_c, s.arec_r, g->stream));
            g->launches += 1;
        }
    }
    PD_CUDA(g, cudaStreamSynchronize(g->stream));
    // cross term present unless K^{xi eta} vanishes identically (orthogonal map, K = d m I,
    // or a separable map with M12 = 0)
    bool separable = s.d.map != PD_MAP_POLAR;
    s.I.has_cross = (c->M12 != 0.0 || (!separable && c->M11 != c->M22)) ? 1 : 0;
    s.coef_set = true;
    for (auto& kv : g->gcache) { cudaGraphExecDestroy(kv.second.exec); cudaGraphDestroy(kv.second.graph); }
    g->gcache.clear();
    return PD_OK;
}

pd_status pd_query(const pd_grid* gc, int inst, pd_info* o)
{
    pd_grid* g = const_cast<pd_grid*>(gc);
    pd_status rc = check_inst(g, inst);
    if (rc) return rc;
    if (!o) return fail(g, PD_EINVAL, "null output");
    const Inst& s = g->inst[inst];
    std::memset(o, 0, sizeof(*o));
    o->n_patch = s.I.n_patch;
    o->n_macro = s.I.nxp * s.I.nyp;
    o->nxp = s.I.nxp; o->nyp = s.I.nyp;
    o->m_xi = s.d.m_xi; o->m_eta = s.d.m_eta; o->k_micro = s.d.k_micro; o->prec = s.d.prec;
    o->u_offset = s.I.u_off;
    o->patch_offset = s.I.p_off;
    o->point_offset = s.I.pt_off;
    o->edge_offset = s.I.e_off;
    o->dt_micro = s.dt; o->tau = s.tau; o->dt_macro_suggested = s.dtm_sugg;
    layout(g, s, *o);
    if (g->q_refresh > 1) o->exec_path = 0;
    else if (use_batch(g)) o->exec_path = all_batch_supported(g) ? 3 : 0;
    else o->exec_path = !fused_supported(s.I) ? 0
                      : (g->persist && s.coef_set && s.I.micro == PD_MICRO_FE && persist_fits(s.I, s.d.prec)) ? 2 : 1;
    o->chunk_steps = o->exec_path == 2 ? persist_max_steps(s.I, s.d.prec) : 1;
    o->has_cross = s.I.has_cross != 0;
    o->has_tsrc = s.I.has_tsrc != 0;
    return PD_OK;
}

pd_status pd_sizes(const pd_grid* g, long long* nm, long long* np, size_t* sb)
{
    if (!g) return PD_EINVAL;
    if (nm) *nm = g->n_macro_total;
    if (np) *np = g->n_patch_total;
    if (sb) *sb = g->state_bytes;
    return PD_OK;
}

pd_status pd_get_coeffs(pd_grid* g, int inst, double* out)
{
    NvtxRange nvtx_range("pd_get_coeffs");
    pd_status rc = check_inst(g, inst);
    if (rc) return rc;
    Inst& s = g->inst[inst];
    if (!s.coef_set) return fail(g, PD_ESTATE, "coefficients not set");
    if (!out) return fail(g, PD_EINVAL, "null output");
    DeviceGuard dg(g->device);
    if (s.I.coef_mode != COEF_RECORDS) PD_CUDA(g, launch_table_get_coeffs(s.I, out, g->stream));
    else PD_CUDA(g, launch_get_coeffs(s.I, s.d.prec, out, g->stream));
    g->launches += 1;
    return PD_OK;
}

pd_status pd_init_field(pd_grid* g, int inst, int kind, const double* prm, int n_prm, double t, double* U)
{
    NvtxRange nvtx_range("pd_init_field");
    pd_status rc = check_inst(g, inst);
    if (rc) return rc;
    Inst& s = g->inst[inst];
    if (!U) return fail(g, PD_EINVAL, "null field");
    if (kind < 0 || kind > 4) return fail(g, PD_EINVAL, "unknown init kind");
    if ((kind == PD_INIT_EXACT) && !s.coef_set) return fail(g, PD_ESTATE, "EXACT needs pd_set_coeffs");
    DeviceGuard dg(g->device);
    double mu[8] = { 0 };
    if (kind == PD_INIT_BESSEL) {
        if (!prm || n_prm < 3 || prm[0] < 1 || prm[0] > 8 || n_prm < 3 + (int)prm[0])
            return fail(g, PD_EINVAL, "BESSEL needs {n_modes<=8, r_in, r_out, a_1..a_n}");
        for (int k = 1; k <= (int)prm[0]; ++k) mu[k - 1] = first_root(k, prm[1], prm[2]);
    }
    if (kind == PD_INIT_ANNULUS_POLY && (!prm || n_prm < 2)) return fail(g, PD_EINVAL, "ANNULUS_POLY needs {r_in, r_out}");
    pd_coeff_desc c = s.coef_set ? s.coef : pd_coeff_desc{};
    if (!s.coef_set) c.d0 = 1.0;
    PD_CUDA(g, launch_init_field(s.I, c, kind, prm, n_prm, mu, t, U + s.I.u_off, g->stream));
    g->launches += 1;
    return PD_OK;
}

pd_status pd_lift(pd_grid* g, const double* U, double t, void* state)
{
    NvtxRange nvtx_range("pd_lift");
    if (!g) return PD_EINVAL;
    if (!U || !state) return fail(g, PD_EINVAL, "null pointer");
    if (((uintptr_t)state) & 255) return fail(g, PD_EINVAL, "state buffer must be 256-byte aligned");
    pd_status rc = all_coeffs_set(g);
    if (rc) return rc;
    DeviceGuard dg(g->device);
    for (auto& s : g->inst) {
        pd_info lay;
        layout(g, s, lay);
        PD_CUDA(g, launch_lift(s.I, nullptr, s.d.prec, U + s.I.u_off, t, (char*)state, lay, g->stream));
        g->launches += 2;
    }
    return PD_OK;
}

pd_status pd_micro_burst(pd_grid* g, void* state, double t, int k_steps)
{
    NvtxRange nvtx_range("pd_micro_burst");
    if (!g) return PD_EINVAL;
    if (!state) return fail(g, PD_EINVAL, "null state");
    if (k_steps < 0 || k_steps > kMaxK) return fail(g, PD_EINVAL, "k_steps must be in [0, 4096]");
    pd_status rc = all_coeffs_set(g);
    if (rc) return rc;
    if (k_steps == 0) return PD_OK;
    DeviceGuard dg(g->device);
    for (auto& s : g->inst)
        if (s.I.micro != PD_MICRO_FE) return fail(g, PD_EINVAL, "the ADI micro solver runs inside pd_step only");
    for (auto& s : g->inst) {
        pd_info lay;
        layout(g, s, lay);
        PD_CUDA(g, launch_burst(s.I, nullptr, s.d.prec, (char*)state, lay, t, k_steps, g->stream));
        g->launches += 2;
    }
    return PD_OK;
}

pd_status pd_restrict(pd_grid* g, const void* state, double* dU)
{
    NvtxRange nvtx_range("pd_restrict");
    if (!g) return PD_EINVAL;
    if (!state || !dU) return fail(g, PD_EINVAL, "null pointer");
    pd_status rc = all_coeffs_set(g);
    if (rc) return rc;
    DeviceGuard dg(g->device);
    for (auto& s : g->inst) {
        pd_info lay;
        layout(g, s, lay);
        PD_CUDA(g, launch_restrict(s.I, s.d.prec, (const char*)state, lay, dU, g->stream));
        g->launches += 1;
    }
    return PD_OK;
}

pd_status pd_project(pd_grid* g, double* U, const double* dU, double t, double dtm)
{
    NvtxRange nvtx_range("pd_project");
    if (!g) return PD_EINVAL;
    if (!U || !dU) return fail(g, PD_EINVAL, "null pointer");
    if (!(dtm > 0)) return fail(g, PD_EINVAL, "dt_macro must be positive");
    pd_status rc = all_coeffs_set(g);
    if (rc) return rc;
    DeviceGuard dg(g->device);
    for (auto& s : g->inst) {
        PD_CUDA(g, launch_project(s.I, U + s.I.u_off, dU, t, dtm, g->stream));
        g->launches += 1;
    }
    return PD_OK;
}

pd_status pd_step(pd_grid* g, double* U, double t0, double dt_macro, int n_macro)
{
    NvtxRange nvtx_range("pd_step");
    if (!g) return PD_EINVAL;
    if (!U) return fail(g, PD_EINVAL, "null field");
    if (n_macro < 0) return fail(g, PD_EINVAL, "n_macro must be >= 0");
    pd_status rc = all_coeffs_set(g);
    if (rc) return rc;
    if (n_macro == 0) return PD_OK;
    DeviceGuard dg(g->device);
    std::vector<double> dtm(g->inst.size());
    for (size_t k = 0; k < g->inst.size(); ++k) dtm[k] = dt_macro > 0 ? dt_macro : g->inst[k].dtm_sugg;
    if (g->q_refresh > 1) {
        if (g->integrator != PD_INT_EULER) return fail(g, PD_EINVAL, "edge refresh runs with the forward-Euler outer step");
        for (auto& s : g->inst)
            if (s.I.coef_mode != COEF_RECORDS || s.I.micro != PD_MICRO_FE || s.I.K % g->q_refresh != 0)
                return fail(g, PD_EINVAL, "edge refresh needs per-point records, forward-Euler bursts and K divisible by q");
        return step_refresh(g, U, t0, dtm, n_macro);
    }
    if (g->integrator != PD_INT_EULER) {
        if (g->inst.size() != 1 || use_batch(g) || !fused_supported(g->inst[0].I))
            return fail(g, PD_EINVAL, "second-order integrators need a grid of one instance with per-point records "
                                      "and m_xi == m_eta in {3,5,7,9,11}");
        return step_higher(g, U, t0, dtm[0], n_macro);
    }
    if (use_batch(g)) {
        if (all_batch_supported(g)) return step_batch(g, U, t0, dtm, n_macro);
        return step_fallback(g, U, t0, dtm, n_macro);
    }
    bool all_fused = true;
    for (auto& s : g->inst) all_fused &= fused_supported(s.I);
    if (!all_fused) return step_fallback(g, U, t0, dtm, n_macro);
    rc = ensure_step_buffers(g, n_macro);
    if (rc) return rc;
    // per-step time tables (s(t) differences, T, T_next) for every instance
    size_t tab_off = 0;
    for (size_t k = 0; k < g->inst.size(); ++k) {
        Inst& s = g->inst[k];
        PD_CUDA(g, launch_time_table(s.I, t0, dtm[k], n_macro, g->tab + tab_off, g->stream));
        g->launches += 1;
        tab_off += (size_t)n_macro * (s.I.K + kTabExtra);
    }
    if (!g->graphs) {
        int nl = 0;
        rc = enqueue_steps(g, U, n_macro, dtm, g->stream, nl);
        g->launches += nl;
        return rc;
    }
    // graphs bake kernel arguments: key on the field pointer, the step count and the macro steps
    GraphKey key{ (uintptr_t)U, n_macro, dtm };
    auto it = g->gcache.find(key);
    if (it == g->gcache.end()) {
        GraphEntry ge;
        PD_CUDA(g, cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal));
        int nl = 0;
        rc = enqueue_steps(g, U, n_macro, dtm, g->cap, nl);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(g->cap, &graph);
        if (rc) { if (graph) cudaGraphDestroy(graph); return rc; }
        if (e != cudaSuccess) return cuda_fail(g, e, "end capture");
        e = cudaGraphInstantiate(&ge.exec, graph, 0);
        if (e != cudaSuccess) { cudaGraphDestroy(graph); return cuda_fail(g, e, "graph instantiate"); }
        ge.graph = graph;
        ge.n_nodes = nl;
        it = g->gcache.emplace(key, ge).first;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (g->timing) {
        for (cudaEvent_t* e : { &e0, &e1 }) {
            if (!g->tfree.empty()) { *e = g->tfree.back(); g->tfree.pop_back(); }
            else PD_CUDA(g, cudaEventCreate(e));
        }
        PD_CUDA(g, cudaEventRecord(e0, g->stream));
    }
    PD_CUDA(g, cudaGraphLaunch(it->second.exec, g->stream));
    g->launches += it->second.n_nodes;
    if (g->timing) {
        PD_CUDA(g, cudaEventRecord(e1, g->stream));
        g->tev.emplace_back(e0, e1);
        g->t_launches += n_macro;
    }
    return PD_OK;
}

pd_status pd_set_coeff_storage(pd_grid* g, int mode)
{
    if (!g) return PD_EINVAL;
    if (mode < 0 || mode > 2) return fail(g, PD_EINVAL, "storage mode must be 0 (auto), 1 (records) or 2 (tables)");
    for (auto& s : g->inst) if (s.coef_set) return fail(g, PD_ESTATE, "set the storage mode before pd_set_coeffs");
    g->storage = mode;
    return PD_OK;
}

pd_status pd_autotune(pd_grid* g, int n_trial_steps, int* block, int* half_patches)
{
    NvtxRange nvtx_range("pd_autotune");
    if (!g) return PD_EINVAL;
    pd_status rc = all_coeffs_set(g);
    if (rc) return rc;
    if (!use_batch(g) || !all_batch_supported(g)) return fail(g, PD_ESTATE, "autotuning applies to batched grids");
    DeviceGuard dg(g->device);
    rc = batch_autotune(g, std::max(1, n_trial_steps));
    if (rc) return rc;
    if (block) *block = g->bt_block;
    if (half_patches) *half_patches = g->bt_half ? 1 : 0;
    return PD_OK;
}

pd_status pd_set_autotune(pd_grid* g, int enabled, int block, int half_patches)
{
    if (!g) return PD_EINVAL;
    if (block != 64 && block != 128) return fail(g, PD_EINVAL, "block must be 64 or 128");
    g->autotune = enabled != 0;
    g->bt_block = block;
    g->bt_half = half_patches != 0;
    g->bt_tuned = false;
    g->batch_dirty = true;
    return PD_OK;
}

pd_status pd_set_integrator(pd_grid* g, int kind)
{
    if (!g) return PD_EINVAL;
    if (kind != PD_INT_EULER && kind != PD_INT_HEUN && kind != PD_INT_AB2) return fail(g, PD_EINVAL, "unknown integrator");
    g->integrator = kind;
    return PD_OK;
}

pd_status pd_set_edge_refresh(pd_grid* g, int q)
{
    if (!g) return PD_EINVAL;
    if (q < 1) return fail(g, PD_EINVAL, "q must be >= 1");
    for (auto& s : g->inst) {
        if (s.I.K % q != 0) return fail(g, PD_EINVAL, "k_micro must be divisible by q");
        if (q > 1 && s.I.micro != PD_MICRO_FE) return fail(g, PD_EINVAL, "edge refresh needs forward-Euler bursts");
    }
    g->q_refresh = q;
    return PD_OK;
}

pd_status pd_set_persistent(pd_grid* g, int enabled)
{
    if (!g) return PD_EINVAL;
    g->persist = enabled != 0;
    for (auto& kv : g->gcache) { cudaGraphExecDestroy(kv.second.exec); cudaGraphDestroy(kv.second.graph); }
    g->gcache.clear();
    return PD_OK;
}

pd_status pd_set_wait_limit(pd_grid* g, long long ns)
{
    if (!g) return PD_EINVAL;
    if (ns < 1000) return fail(g, PD_EINVAL, "wait limit below 1 us");
    g->wait_ns = ns;
    for (auto& kv : g->gcache) { cudaGraphExecDestroy(kv.second.exec); cudaGraphDestroy(kv.second.graph); }
    g->gcache.clear();
    return PD_OK;
}

pd_status pd_test_silence_warp(pd_grid* g, int warp)
{
    if (!g) return PD_EINVAL;
    g->silent_warp = warp;
    for (auto& kv : g->gcache) { cudaGraphExecDestroy(kv.second.exec); cudaGraphDestroy(kv.second.graph); }
    g->gcache.clear();
    return PD_OK;
}

pd_status pd_set_timing(pd_grid* g, int enabled)
{
    if (!g) return PD_EINVAL;
    double ms;
    long long n;
    pd_get_timing(g, &ms, &n);
    g->timing = enabled != 0;
    g->t_ms = 0.0;
    g->t_launches = 0;
    return PD_OK;
}

pd_status pd_get_timing(pd_grid* g, double* ms, long long* n)
{
    if (!g) return PD_EINVAL;
    for (auto& pr : g->tev) {
        PD_CUDA(g, cudaEventSynchronize(pr.second));
        float f = 0.f;
        PD_CUDA(g, cudaEventElapsedTime(&f, pr.first, pr.second));
        g->t_ms += f;
        g->tfree.push_back(pr.first);
        g->tfree.push_back(pr.second);
    }
    g->tev.clear();
    if (ms) *ms = g->t_ms;
    if (n) *n = g->t_launches;
    return PD_OK;
}

pd_status pd_sync(pd_grid* g)
{
    NvtxRange nvtx_range("pd_sync");
    if (!g) return PD_EINVAL;
    DeviceGuard dg(g->device);
    PD_CUDA(g, cudaStreamSynchronize(g->stream));
    int h = 0;
    PD_CUDA(g, cudaMemcpy(&h, g->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (h & ERR_TIMEOUT) {
        cudaMemset(g->err, 0, sizeof(int));
        return fail(g, PD_ETIMEOUT, "a patch warp gave up waiting for its neighbours' macro step");
    }
    if (h & ERR_NONFINITE) {
        cudaMemset(g->err, 0, sizeof(int));
        return fail(g, PD_ENUMERIC, "non-finite restricted change (unstable macro or micro step?)");
    }
    return PD_OK;
}

namespace {
uint64_t desc_hash(const pd_grid* g)
{
    uint64_t h = 1469598103934665603ull;
    for (auto& s : g->inst) {
        const unsigned char* p = reinterpret_cast<const unsigned char*>(&s.d);
        for (size_t k = 0; k < sizeof(s.d); ++k) { h ^= p[k]; h *= 1099511628211ull; }
    }
    return h;
}
const char kMagic[8] = { 'P', 'D', 'C', 'K', 'P', 'T', '0', '1' };
}  // namespace

pd_status pd_save_checkpoint(pd_grid* g, const double* U, double t, long long step, const char* path)
{
    NvtxRange nvtx_range("pd_save_checkpoint");
    if (!g || !U || !path) return fail(g, PD_EINVAL, "null argument");
    DeviceGuard dg(g->device);
    std::vector<double> h((size_t)g->n_macro_total);
    PD_CUDA(g, cudaMemcpyAsync(h.data(), U, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, g->stream));
    PD_CUDA(g, cudaStreamSynchronize(g->stream));
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(g, PD_EINVAL, std::string("cannot open ") + path);
    uint64_t hash = desc_hash(g);
    long long n = g->n_macro_total;
    bool ok = std::fwrite(kMagic, 1, 8, f) == 8 && std::fwrite(&hash, 8, 1, f) == 1 && std::fwrite(&n, 8, 1, f) == 1
           && std::fwrite(&t, 8, 1, f) == 1 && std::fwrite(&step, 8, 1, f) == 1
           && std::fwrite(h.data(), sizeof(double), h.size(), f) == h.size();
    ok &= std::fclose(f) == 0;
    return ok ? PD_OK : fail(g, PD_EINVAL, "short write");
}

pd_status pd_load_checkpoint(pd_grid* g, double* U, double* t, long long* step, const char* path)
{
    NvtxRange nvtx_range("pd_load_checkpoint");
    if (!g || !U || !path) return fail(g, PD_EINVAL, "null argument");
    DeviceGuard dg(g->device);
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(g, PD_EINVAL, std::string("cannot open ") + path);
    char mg[8];
    uint64_t hash = 0;
    long long n = 0, st = 0;
    double tt = 0;
    bool ok = std::fread(mg, 1, 8, f) == 8 && std::fread(&hash, 8, 1, f) == 1 && std::fread(&n, 8, 1, f) == 1
           && std::fread(&tt, 8, 1, f) == 1 && std::fread(&st, 8, 1, f) == 1;
    if (!ok || std::memcmp(mg, kMagic, 8) != 0) { std::fclose(f); return fail(g, PD_EINVAL, "not a checkpoint"); }
    if (hash != desc_hash(g) || n != g->n_macro_total) { std::fclose(f); return fail(g, PD_EINVAL, "checkpoint of another grid"); }
    std::vector<double> h((size_t)n);
    ok = std::fread(h.data(), sizeof(double), h.size(), f) == h.size();
    std::fclose(f);
    if (!ok) return fail(g, PD_EINVAL, "truncated checkpoint");
    PD_CUDA(g, cudaMemcpyAsync(U, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice, g->stream));
    PD_CUDA(g, cudaStreamSynchronize(g->stream));
    if (t) *t = tt;
    if (step) *step = st;
    return PD_OK;
}

}  // extern "C"

namespace pd {

pd_status grid_access(pd_grid* g, int inst, GridAccess& out)
{
    if (!g) return PD_EINVAL;
    if (inst < 0 || inst >= (int)g->inst.size()) return fail(g, PD_EINVAL, "instance index out of range");
    const Inst& s = g->inst[inst];
    if (!s.coef_set) return fail(g, PD_ESTATE, "coefficients not set");
    out.I = s.I;
    out.coef = s.coef;
    out.prec = s.d.prec;
    out.n_inst = (int)g->inst.size();
    out.device = g->device;
    out.stream = g->stream;
    out.dtm_sugg = s.dtm_sugg;
    return PD_OK;
}

void grid_message(pd_grid* g, const char* msg)
{
    if (g) g->last = msg;
}

void grid_count_launches(pd_grid* g, long long n)
{
    if (g) g->launches += n;
}

}  // namespace pd

// ---------------------------------------------------------------------------
// pd_step_noalloc: the fused per-step path of pd_step with both of its scratch
// buffers (the second macro field and the per-step time table) carved out of
// one fixed device array instead of device allocations.

namespace {

constexpr size_t kNoAllocDoubles = size_t(1) << 19;   // 4 MiB per device

static __device__ __align__(256) double noalloc_scratch[kNoAllocDoubles];

// Device address of the array in the current context of the grid's device
// (the caller holds a DeviceGuard for it).  In host code the array's name is
// only a host-side stand-in, so kernels get this address instead.  It is looked
// up on every call rather than cached: a context torn down and created again
// (cudaDeviceReset) loads the module at another address.  The first lookup in
// a context loads the module (set-up work in the CUDA runtime).
pd_status noalloc_scratch_on(pd_grid* g, double** out)
{
    void* p = nullptr;
    PD_CUDA(g, cudaGetSymbolAddress(&p, noalloc_scratch));
    *out = static_cast<double*>(p);
    return PD_OK;
}

}  // namespace

extern "C" {

pd_status pd_step_noalloc(pd_grid* g, double* U, double t0, double dt_macro, int n_macro)
{
    NvtxRange nvtx_range("pd_step_noalloc");
    if (!g) return PD_EINVAL;
    if (!U) return fail(g, PD_EINVAL, "null field");
    if (n_macro < 0) return fail(g, PD_EINVAL, "n_macro must be >= 0");
    pd_status rc = all_coeffs_set(g);
    if (rc) return rc;
    if (g->inst.size() != 1) return fail(g, PD_EINVAL, "pd_step_noalloc takes a grid of one instance");
    if (g->integrator != PD_INT_EULER)
        return fail(g, PD_EINVAL, "pd_step_noalloc runs the forward-Euler outer step only (pd_set_integrator)");
    if (g->q_refresh > 1)
        return fail(g, PD_EINVAL, "pd_step_noalloc keeps the edge data fixed over a burst (pd_set_edge_refresh q = 1)");
    Inst& s = g->inst[0];
    const InstDev& I = s.I;
    if (I.coef_mode != COEF_RECORDS || !fused_supported(I))
        return fail(g, PD_EINVAL, "pd_step_noalloc needs per-point coefficient records and m_xi == m_eta in {3,5,7,9,11}");
    // layout: second macro field (rounded to 256 bytes), then n_macro time-table rows
    const size_t field = ((size_t)I.nxp * I.nyp + 31) & ~size_t(31);
    const size_t stride = (size_t)I.K + kTabExtra;
    const size_t need = field + (size_t)n_macro * stride;
    if (need > kNoAllocDoubles)
        return fail(g, PD_EINVAL, "pd_step_noalloc needs " + std::to_string(need) +
                                  " doubles of fixed scratch (field + n_macro time-table rows); the limit is " +
                                  std::to_string(kNoAllocDoubles) + ": take fewer macro steps per call");
    if (n_macro == 0) return PD_OK;
    DeviceGuard dg(g->device);
    double* base = nullptr;
    rc = noalloc_scratch_on(g, &base);
    if (rc) return rc;
    const double dtm = dt_macro > 0 ? dt_macro : s.dtm_sugg;
    double* tab = base + field;
    PD_CUDA(g, launch_time_table(I, t0, dtm, n_macro, tab, g->stream));
    int nl = 1;
    double* bufs[2] = { U + I.u_off, base };
    for (int t = 0; t < n_macro; ++t) {
        cudaError_t e = launch_fused_step(I, nullptr, s.d.prec, bufs[t & 1], bufs[(t + 1) & 1],
                                          tab + (size_t)t * stride, dtm, g->stream, &nl);
        if (e != cudaSuccess) { g->launches += nl; return cuda_fail(g, e, "fused step (fixed scratch)"); }
    }
    g->launches += nl;
    if (n_macro & 1)
        PD_CUDA(g, cudaMemcpyAsync(bufs[0], bufs[1], sizeof(double) * (size_t)I.nxp * I.nyp,
                                   cudaMemcpyDeviceToDevice, g->stream));
    return PD_OK;
}

}  // extern "C"

// Host runtime of libepr: plans, device workspace, the C ABI of include/epr.h,
// launch sequences of the solvers and their capture in CUDA graphs.
//
// One solver iteration (arXiv 2601.22793, "Iterative inversion") is four
// kernels over the whole batch:
//   splat     forward transport of all lines, P and P_s        (splat.cu)
//   row_fwd   split + adjoint gather + R2C row FFT, rho share  (rowfft.cu)
//   col       column FFT, Paganin filter, inverse column FFT   (colfft.cu)
//   row_inv   C2R row FFT + update + projection, kappa share   (rowfft.cu)
// The local solver replaces splat by the stencil closure (local.cu) and the
// gather by the identity.  The iteration loop is captured once per
// (buffers, batch, options) into a CUDA graph and replayed.
#include <math.h>
#include <stdio.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <new>
#include <type_traits>
#include <vector>

#include <cuda.h>

#include "epr_internal.cuh"

// --- launchers from the other translation units -----------------------------
cudaError_t epr_launch_splat(const EprConsts& C, const EprWork& W, const float* T, const float* D,
                             int resid, int parity, int batch, int TH, int TW, int check_done,
                             cudaStream_t stream);
size_t epr_splat_smem(const EprConsts& C, int TH, int TW);
bool epr_splat_has_occ6(int TH, int TW, int reach);
cudaError_t epr_splat_init();
cudaError_t epr_launch_row_fwd(const EprConsts& C, const EprWork& W, int mode, const float* T,
                               const float* D, const float* G, int line0, int nl, int it,
                               float tol, int batch, int check_done, cudaStream_t stream);
cudaError_t epr_launch_split(const EprConsts& C, const EprWork& W, const float* D, int batch,
                             int fixed_point, int check_done, cudaStream_t stream);
cudaError_t epr_launch_dnorm(const EprConsts& C, const EprWork& W, const float* D, int batch,
                             size_t npix, double scale, cudaStream_t stream);
cudaError_t epr_launch_split_os(const EprConsts& C, const EprWork& W, const float* D, int batch,
                                int fixed_point, int check_done, cudaStream_t stream);
cudaError_t epr_launch_bin_os(const EprConsts& C, const EprWork& W, int fixed_point, float* out,
                              float* outs, int batch, cudaStream_t stream);
cudaError_t epr_launch_row_inv(const EprConsts& C, const EprWork& W, int mode, float* Out, int line0,
                               int nl, int it, float omega, float eps, float tol, int batch,
                               int check_done, cudaStream_t stream);
cudaError_t epr_row_init();
bool epr_col_make_map(const EprConsts& C, const float2* S, long long rows, CUtensorMap* out);
cudaError_t epr_launch_col(const EprConsts& C, const EprWork& W, int line0, int nl, int batch,
                           int check_done, int cw_hint, int rho_it, cudaStream_t stream);
cudaError_t epr_launch_finalize_kappa(const EprConsts& C, const EprWork& W, int it, float tol,
                                      int batch, cudaStream_t stream);
cudaError_t epr_col_init();
cudaError_t epr_launch_gather(const EprConsts& C, const float* T, const float* r, float* g, int line,
                              int batch, cudaStream_t stream);
cudaError_t epr_launch_fx_to_float(const unsigned long long* q, float* out, size_t n, cudaStream_t stream);
cudaError_t epr_launch_local(const EprConsts& C, const EprWork& W, const float* T, float* P, float* Ps,
                             int order, int batch, int check_done, cudaStream_t stream);
cudaError_t epr_local_init();
cudaError_t epr_launch_wkb1(const EprConsts& C, const EprWork& W, const float* T, int fixed_point,
                            int batch, int check_done, cudaStream_t stream);
cudaError_t epr_launch_col_kind(const EprConsts& C, const EprWork& W, int line, int batch, int kind,
                                float kscale, cudaStream_t stream);
int epr_sv_blocks();
cudaError_t epr_launch_sv_split(const EprConsts& C, const float* D, const float* P, const float* Ps,
                                float* r, float* RS, int B, cudaStream_t s);
cudaError_t epr_launch_sv_update_adj(const EprConsts& C, const float* T, const float* Hs, const float* tb,
                                     float* HB, double* part, int B, float omega, float eps,
                                     float inv_den, cudaStream_t s);
cudaError_t epr_launch_sv_dot(const float* a, const float* b, size_t npix, double* part, int B,
                              cudaStream_t s);
cudaError_t epr_launch_sv_splat_field(const EprConsts& C, const float* T, const float* field, float* out,
                                      int line, int B, cudaStream_t s);
cudaError_t epr_launch_sv_interp_du(const EprConsts& C, int mode, const float* T, const float* e,
                                    const float* wmap, const float* HB, float* vx, float* vy, float* tn,
                                    double* part, int line, float omega, int B, cudaStream_t s);
cudaError_t epr_launch_sv_split_adj(const EprConsts& C, float* RSB, const float* P, const float* Ps,
                                    const float* r, float* Db, int B, cudaStream_t s);
cudaError_t epr_launch_sv_gT(const EprConsts& C, const float* vx, const float* vy, float* tn, int B,
                             cudaStream_t s);
cudaError_t epr_launch_sv_accum(const double* part, size_t npix, int nslot, int slot, double* acc,
                                int nacc, int slot_acc, double scale, int B, cudaStream_t s);
cudaError_t epr_launch_vjp(const EprConsts& C, const float* T, const float* gbar, float* Tbar,
                           float* vx, float* vy, double* part, int nblk, int batch,
                           cudaStream_t stream);

// --- launch accounting -------------------------------------------------------
static std::atomic<long long> g_launches(0);
void epr_count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
extern "C" long long epr_launch_count(void) { return g_launches.load(); }

// --- plan --------------------------------------------------------------------
namespace {

constexpr double kHcEvM = 1.2398419843320026e-6;  // h c in eV m
constexpr double kPi = 3.14159265358979323846;

struct GraphKey {
    const void* D;
    const void* T;
    int batch, n_iter, init, model;
    double omega, tol, eps;
    bool operator==(const GraphKey& o) const
    {
        return D == o.D && T == o.T && batch == o.batch && n_iter == o.n_iter && init == o.init &&
               model == o.model && omega == o.omega && tol == o.tol && eps == o.eps;
    }
};

}  // namespace

struct epr_plan_s {
    EprConsts C;
    epr_options opt;
    int device;
    double pixel, L;
    double E[EPR_MAX_LINES], delta[EPR_MAX_LINES], beta[EPR_MAX_LINES], w[EPR_MAX_LINES];
    // workspace
    EprWork W;
    alignas(64) CUtensorMap col_map;   // S for the column pass's bulk copies
    int cap_batch;       // batch the workspace is sized for
    int cap_hist;        // history length it is sized for
    std::vector<void*> allocs;
    float2* tw_x;
    float2* tw_y;
    // staging of host arrays
    float* stage[3];
    size_t stage_elems[3];
    // pinned host copies for solve info
    EprProjState* h_st;
    double* h_hist;
    size_t h_hist_elems;
    // tiles
    int splat_TH, splat_TW;
    int col_cw;          // column tile width of the solver's column pass (0 = default)
    // kernel timing (benchmarks)
    bool profiling;
    struct Rec {
        int kind;
        cudaEvent_t a, b;
    };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    // graph cache
    cudaStream_t cap_stream;
    cudaGraphExec_t gexec;
    GraphKey gkey;
    int gkernels;
    bool has_graph;
    cudaGraphExec_t prof_exec;   // last profiled solve
    bool tuned;                  // autotuner has run
    // vector-Jacobian product workspace (allocated on first use)
    float* vjp_vx;
    float* vjp_vy;
    double* vjp_part;
    double* h_vjp_part;
    int vjp_cap;
    // x-dependent spectrum: per-column constants on the device (C.xt points
    // here while a table is set) and the uniform preconditioner constants
    float* xt_dev;
    float ha_uniform[EPR_MAX_LINES], hb_uniform[EPR_MAX_LINES];
    // reverse mode through the solve (allocated on first use, kept for reuse)
    std::vector<void*> sv_allocs;
    int sv_batch, sv_nck, sv_nseg;
    float *sv_r, *sv_RS, *sv_GA, *sv_H, *sv_HB, *sv_GB, *sv_TMP, *sv_RSB;
    float *sv_tb, *sv_tn, *sv_vx, *sv_vy, *sv_Db, *sv_ck, *sv_seg;
    double *sv_part, *sv_acc, *h_sv_acc;
};

namespace {

// 2^a 3^b with a >= 3, from 16 to nmax (4096; 8192 for an oversampled
// internal grid)
bool size_ok(int n, int nmax = 4096)
{
    if (n < 16 || n > nmax) return false;
    int m = n, twos = 0;
    while (m % 2 == 0) {
        m /= 2;
        ++twos;
    }
    while (m % 3 == 0) m /= 3;
    return m == 1 && twos >= 3;
}

epr_status cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return EPR_OK;
    if (e == cudaErrorMemoryAllocation) return EPR_ERR_OOM;
    return EPR_ERR_CUDA;
}

#define EPR_TRY(expr)                                       \
    do {                                                    \
        cudaError_t _e = (expr);                            \
        if (_e != cudaSuccess) return cuda_status(_e);      \
    } while (0)

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

bool is_device_ptr(const void* p)
{
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void free_workspace(epr_plan_s* p)
{
    for (void* a : p->allocs) cudaFree(a);
    p->allocs.clear();
    // tuner choices
    const int radix16 = p->W.col_radix16, occ6 = p->W.row_occ6, cocc5 = p->W.col_occ5;
    const int socc6 = p->W.splat_occ6;
    memset(&p->W, 0, sizeof(p->W));
    p->W.col_radix16 = radix16;
    p->W.row_occ6 = occ6;
    p->W.col_occ5 = cocc5;
    p->W.splat_occ6 = socc6;
    p->W.tw_x = p->tw_x;
    p->W.tw_y = p->tw_y;
    p->cap_batch = 0;
    p->cap_hist = 0;
    if (p->has_graph) {
        cudaGraphExecDestroy(p->gexec);
        p->has_graph = false;
    }
}

template <typename T>
cudaError_t dalloc(epr_plan_s* p, T** out, size_t n)
{
    void* ptr = nullptr;
    cudaError_t e = cudaMalloc(&ptr, n * sizeof(T) > 0 ? n * sizeof(T) : 16);
    if (e != cudaSuccess) return e;
    p->allocs.push_back(ptr);
    *out = reinterpret_cast<T*>(ptr);
    return cudaSuccess;
}

epr_status ensure_workspace(epr_plan_s* p, int batch, int hist)
{
    if (batch <= p->cap_batch && hist <= p->cap_hist && p->cap_batch > 0) return EPR_OK;
    const int nb = batch > p->cap_batch ? batch : p->cap_batch;
    const int nh = hist > p->cap_hist ? hist : (p->cap_hist > 0 ? p->cap_hist : 1);
    cudaDeviceSynchronize();
    free_workspace(p);
    const EprConsts& C = p->C;
    const size_t npix = (size_t)C.nx * C.ny;
    EprWork& W = p->W;
    cudaError_t e = cudaSuccess;
    W.max_blocks = C.ny / 2;
    W.hist_len = nh;
    e = dalloc(p, &W.P, (size_t)nb * npix);
    if (e == cudaSuccess && C.ns > 1) e = dalloc(p, &W.Ps, (size_t)nb * C.ns * npix);
    if (e == cudaSuccess && C.det) e = dalloc(p, &W.Pq, (size_t)nb * npix);
    if (e == cudaSuccess && C.det && C.ns > 1) e = dalloc(p, &W.Psq, (size_t)nb * C.ns * npix);
    if (e == cudaSuccess) e = dalloc(p, &W.S, (size_t)nb * C.ns * C.ny * C.half);
    if (e == cudaSuccess) e = dalloc(p, &W.ovf_idx, (size_t)nb * C.ovf_cap);
    if (e == cudaSuccess) e = dalloc(p, &W.ovf_mask, (size_t)nb * C.ovf_cap);
    if (e == cudaSuccess) e = dalloc(p, &W.ovf_tg, (size_t)nb * C.ovf_cap);
    if (e == cudaSuccess) e = dalloc(p, &W.st, (size_t)nb);
    if (e == cudaSuccess) e = dalloc(p, &W.part_a, (size_t)nb * W.max_blocks);
    if (e == cudaSuccess) e = dalloc(p, &W.part_b, (size_t)nb * W.max_blocks);
    if (e == cudaSuccess) e = dalloc(p, &W.part_c, (size_t)nb * W.max_blocks);
    if (e == cudaSuccess) e = dalloc(p, &W.rho_hist, (size_t)nb * nh);
    if (e == cudaSuccess) e = dalloc(p, &W.kappa_hist, (size_t)nb * nh);
    if (e == cudaSuccess) e = dalloc(p, &W.err, 1);
    if (e == cudaSuccess) e = cudaMemset(W.st, 0, (size_t)nb * sizeof(EprProjState));
    if (e == cudaSuccess) e = cudaMemset(W.err, 0, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(W.rho_hist, 0, (size_t)nb * nh * sizeof(double));
    if (e == cudaSuccess) e = cudaMemset(W.kappa_hist, 0, (size_t)nb * nh * sizeof(double));
    if (e != cudaSuccess) {
        free_workspace(p);
        return cuda_status(e);
    }
    W.tw_x = p->tw_x;
    W.tw_y = p->tw_y;
    if (p->opt.fft_radix == 16) W.col_radix16 = 1;
    W.col_map = epr_col_make_map(C, W.S, (long long)nb * C.ns * C.ny, &p->col_map) ? &p->col_map
                                                                                   : nullptr;
    p->cap_batch = nb;
    p->cap_hist = nh;
    // pinned host mirrors for solve info
    if (p->h_st) cudaFreeHost(p->h_st);
    if (p->h_hist) cudaFreeHost(p->h_hist);
    p->h_st = nullptr;
    p->h_hist = nullptr;
    e = cudaMallocHost((void**)&p->h_st, (size_t)nb * sizeof(EprProjState));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&p->h_hist, (size_t)2 * nb * nh * sizeof(double));
    if (e != cudaSuccess) return cuda_status(e);
    p->h_hist_elems = (size_t)2 * nb * nh;
    return EPR_OK;
}

// Device view of a caller array: the pointer itself, or a staging buffer
// (filled from the host when `copy_in`).
epr_status resolve(epr_plan_s* p, int slot, const float* ptr, size_t n, bool copy_in,
                   cudaStream_t s, float** out, bool* staged)
{
    if (is_device_ptr(ptr)) {
        *out = const_cast<float*>(ptr);
        *staged = false;
        return EPR_OK;
    }
    if (p->stage_elems[slot] < n) {
        if (p->stage[slot]) {
            cudaStreamSynchronize(s);
            cudaFree(p->stage[slot]);
            p->stage[slot] = nullptr;
        }
        EPR_TRY(cudaMalloc((void**)&p->stage[slot], n * sizeof(float)));
        p->stage_elems[slot] = n;
        if (p->has_graph) {  // staging address changed: the cached graph is stale
            cudaGraphExecDestroy(p->gexec);
            p->has_graph = false;
        }
    }
    if (copy_in) EPR_TRY(cudaMemcpyAsync(p->stage[slot], ptr, n * sizeof(float), cudaMemcpyHostToDevice, s));
    *out = p->stage[slot];
    *staged = true;
    return EPR_OK;
}

void choose_splat_tiles(epr_plan_s* p)
{
    const EprConsts& C = p->C;
    const int cand[3][2] = {{64, 64}, {32, 64}, {32, 32}};
    p->splat_TH = 32;
    p->splat_TW = 32;
    for (auto& c : cand) {
        const size_t acc = (size_t)C.ns * c[0] * c[1] * (C.det ? 8 : 4);
        if (acc <= 65536 && epr_splat_smem(C, c[0], c[1]) <= 200 * 1024) {
            p->splat_TH = c[0];
            p->splat_TW = c[1];
            break;
        }
    }
}

// Events come from a pool filled when profiling is enabled (none is created
// while a stream is being captured); an empty pool skips the timing.
constexpr int kProfEvents = 8192;

cudaEvent_t pool_get(epr_plan_s* p)
{
    if (p->pool.empty()) return nullptr;
    cudaEvent_t e = p->pool.back();
    p->pool.pop_back();
    return e;
}

// Brackets one kernel launch with events when the plan is profiling.
struct ProfScope {
    epr_plan_s* p;
    cudaStream_t s;
    int kind;
    cudaEvent_t a = nullptr;
    ProfScope(epr_plan_s* p_, int kind_, cudaStream_t s_) : p(p_), s(s_), kind(kind_)
    {
        if (p->profiling) {
            a = pool_get(p);
            if (a) cudaEventRecordWithFlags(a, s, cudaEventRecordExternal);
        }
    }
    ~ProfScope()
    {
        if (!a) return;
        cudaEvent_t b = pool_get(p);
        if (!b) {
            p->pool.push_back(a);
            return;
        }
        cudaEventRecordWithFlags(b, s, cudaEventRecordExternal);
        p->recs.push_back({kind, a, b});
    }
};

// One pass of the chosen forward model writing W.P (and W.Ps / W.Pq / W.Psq).
// With D given (monochromatic float solve) W.P receives D - P instead of P.
epr_status launch_forward(epr_plan_s* p, const float* T, const float* D, int parity, int batch,
                          int model, int check_done, cudaStream_t s)
{
    if (model == EPR_MODEL_NONLOCAL || model == EPR_MODEL_NONLOCAL_WKB1) {
        {
            ProfScope ps(p, EPR_KERNEL_SPLAT, s);
            EPR_TRY(epr_launch_splat(p->C, p->W, T, D, D != nullptr, parity, batch, p->splat_TH,
                                     p->splat_TW, check_done, s));
        }
        if (model == EPR_MODEL_NONLOCAL_WKB1) {   // second-order term: float P, P_s after it
            ProfScope ps(p, EPR_KERNEL_LOCAL, s);
            EPR_TRY(epr_launch_wkb1(p->C, p->W, T, p->C.det, batch, check_done, s));
        }
    } else {
        ProfScope ps(p, EPR_KERNEL_LOCAL, s);
        EPR_TRY(epr_launch_local(p->C, p->W, T, p->W.P, p->W.Ps, model, batch, check_done, s));
    }
    return EPR_OK;
}

// The whole solve, launched on stream s (captured or not).
epr_status launch_solve(epr_plan_s* p, const float* D, float* T, int batch, const epr_solve_opts* o,
                        int model, cudaStream_t s)
{
    const EprConsts& C = p->C;
    const size_t npix = (size_t)C.nx * C.ny;
    EPR_TRY(cudaMemsetAsync(p->W.st, 0, (size_t)batch * sizeof(EprProjState), s));
    EPR_TRY(cudaMemsetAsync(p->W.err, 0, sizeof(unsigned int), s));
    if (o->init == 0) EPR_TRY(cudaMemsetAsync(T, 0, (size_t)batch * npix * sizeof(float), s));
    {
        ProfScope ps(p, EPR_KERNEL_OTHER, s);
        // |D|^2 at detector resolution; with oversampling the norm of the
        // residual is taken over its o^2-fold replication, so scale by o^2
        const size_t npd = npix / ((size_t)C.os * C.os);
        EPR_TRY(epr_launch_dnorm(C, p->W, D, batch, npd, (double)C.os * C.os, s));
    }
    // the non-local models back-transport with the gather, the local closures
    // with the identity
    const bool nonlocal = model == EPR_MODEL_NONLOCAL || model == EPR_MODEL_NONLOCAL_WKB1;
    const int fwd_mode = nonlocal ? 0 : 1;
    // the residual D - P (and its split over the lines) is stored by the
    // splat flush (plain non-local model, one line, float accumulation) or by
    // the split kernel after the forward (several lines, fixed point, local
    // closure, second-order non-local model)
    const bool nl = model == EPR_MODEL_NONLOCAL;   // P still in the splat's own format
    const bool resid_in_splat = nl && C.ns == 1 && !C.det && C.os == 1 && !C.xt;
    const float eps = (float)(o->eps_I > 0 ? o->eps_I : 1e-8);
    for (int it = 0; it < o->n_iter; ++it) {
        epr_status st = launch_forward(p, T, resid_in_splat ? D : nullptr, it & 1, batch, model, 1, s);
        if (st != EPR_OK) return st;
        if (C.os > 1) {
            ProfScope ps(p, EPR_KERNEL_OTHER, s);
            EPR_TRY(epr_launch_split_os(C, p->W, D, batch, nl && C.det, 1, s));
        } else if (!resid_in_splat) {
            ProfScope ps(p, EPR_KERNEL_OTHER, s);
            EPR_TRY(epr_launch_split(C, p->W, D, batch, nl && C.det, 1, s));
        }
        {
            ProfScope ps(p, EPR_KERNEL_ROW_FWD, s);
            EPR_TRY(epr_launch_row_fwd(C, p->W, fwd_mode, T, D, nullptr, 0, C.ns, it,
                                       (float)o->tol, batch, 1, s));
        }
        {
            ProfScope ps(p, EPR_KERNEL_COL, s);
            EPR_TRY(epr_launch_col(C, p->W, 0, C.ns, batch, 1, p->col_cw, it, s));
        }
        {
            ProfScope ps(p, EPR_KERNEL_ROW_INV, s);
            EPR_TRY(epr_launch_row_inv(C, p->W, 0, T, 0, C.ns, it, (float)o->omega, eps,
                                       (float)o->tol, batch, 1, s));
        }
    }
    if (o->n_iter > 0) {   // kappa of the last iteration (the others: each next forward pass)
        ProfScope ps(p, EPR_KERNEL_OTHER, s);
        EPR_TRY(epr_launch_finalize_kappa(C, p->W, o->n_iter - 1, (float)o->tol, batch, s));
    }
    return EPR_OK;
}

// Per-projection results of the last solve of plan p (batch projections),
// written at offset `first` of the caller's arrays.  Synchronises s.
epr_status collect_info(epr_plan_s* p, int batch, int n_iter, epr_solve_info* info, cudaStream_t s,
                        int first)
{
    const int nh = p->W.hist_len;
    EPR_TRY(cudaMemcpyAsync(p->h_st, p->W.st, (size_t)batch * sizeof(EprProjState),
                            cudaMemcpyDeviceToHost, s));
    EPR_TRY(cudaMemcpyAsync(p->h_hist, p->W.rho_hist, (size_t)batch * nh * sizeof(double),
                            cudaMemcpyDeviceToHost, s));
    EPR_TRY(cudaMemcpyAsync(p->h_hist + (size_t)batch * nh, p->W.kappa_hist,
                            (size_t)batch * nh * sizeof(double), cudaMemcpyDeviceToHost, s));
    unsigned int herr = 0;
    EPR_TRY(cudaMemcpyAsync(&herr, p->W.err, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
    EPR_TRY(cudaStreamSynchronize(s));
    long long ovf = 0;
    for (int b = 0; b < batch; ++b) {
        const EprProjState& ps = p->h_st[b];
        const int k = ps.iters;
        const int j = first + b;
        if (info->iters) info->iters[j] = k;
        if (info->rho) info->rho[j] = k > 0 ? p->h_hist[(size_t)b * nh + k - 1] : 0.0;
        if (info->kappa) info->kappa[j] = k > 0 ? p->h_hist[(size_t)(batch + b) * nh + k - 1] : 0.0;
        for (int i = 0; i < n_iter; ++i) {
            const bool ran = i < k;
            if (info->rho_hist)
                info->rho_hist[(size_t)j * n_iter + i] = ran ? p->h_hist[(size_t)b * nh + i] : 0.0;
            if (info->kappa_hist)
                info->kappa_hist[(size_t)j * n_iter + i] =
                    ran ? p->h_hist[(size_t)(batch + b) * nh + i] : 0.0;
        }
        ovf += ps.ovf_total;
    }
    if (first == 0) info->overflow_sources = 0;
    info->overflow_sources += ovf;
    if (herr & EPR_DEVERR_NONFINITE) return EPR_ERR_NONFINITE;
    if (herr & EPR_DEVERR_TIMEOUT) return EPR_ERR_TIMEOUT;
    if (herr & EPR_DEVERR_OVERFLOW) return EPR_ERR_SHIFT_OVERFLOW;
    return EPR_OK;
}

// Times the splat's tile shapes and reach (and, where the one-line residual
// kernel has the variant, five or six blocks per SM) on the thickness T of
// the solve that just ran (the real shift field), keeps the fastest and
// drops the cached graph.  Changes only the float summation order of the
// splat.
epr_status autotune_splat(epr_plan_s* p, const float* D, const float* T, int batch, cudaStream_t s)
{
    p->tuned = true;
    const bool resid = p->C.ns == 1 && !p->C.det && p->C.os == 1 && !p->C.xt;
    const int tiles[4][2] = {{64, 64}, {32, 64}, {64, 32}, {32, 32}};
    // the compile-time reaches, and the plan's own when it is none of them
    const int own = p->C.smax;
    const int reaches[4] = {3, 4, 6, (own == 3 || own == 4 || own == 6) ? 0 : own};
    const EprConsts saved = p->C;
    const int sTH = p->splat_TH, sTW = p->splat_TW;
    int optin = 0;
    EPR_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device));
    float best = 1e30f;
    int bTH = sTH, bTW = sTW, bR = saved.smax, bO = p->W.splat_occ6;
    cudaEvent_t e0, e1;
    EPR_TRY(cudaEventCreate(&e0));
    EPR_TRY(cudaEventCreate(&e1));
    for (const auto& t : tiles) {
        for (int r : reaches) for (int occ6 = 0; occ6 <= 1; ++occ6) {
            if (r == 0) continue;
            if (occ6 && !(resid && epr_splat_has_occ6(t[0], t[1], r))) continue;
            p->C.smax = r;
            if ((size_t)p->C.ns * t[0] * t[1] * (p->C.det ? 8 : 4) > 65536) continue;
            if (epr_splat_smem(p->C, t[0], t[1]) + 4096 > (size_t)optin) continue;
            p->splat_TH = t[0];
            p->splat_TW = t[1];
            p->W.splat_occ6 = occ6;
            EPR_TRY(cudaMemsetAsync(p->W.st, 0, (size_t)batch * sizeof(EprProjState), s));
            epr_status st = launch_forward(p, T, resid ? D : nullptr, 0, batch, EPR_MODEL_NONLOCAL, 0, s);
            if (st != EPR_OK) return st;
            float ms = 1e30f;   // the fastest of three repetitions of four forwards
            for (int rep = 0; rep < 3; ++rep) {
                EPR_TRY(cudaEventRecord(e0, s));
                for (int k = 0; k < 4; ++k) {
                    st = launch_forward(p, T, resid ? D : nullptr, (k + 1) & 1, batch, EPR_MODEL_NONLOCAL,
                                        0, s);
                    if (st != EPR_OK) return st;
                }
                EPR_TRY(cudaEventRecord(e1, s));
                EPR_TRY(cudaEventSynchronize(e1));
                float r_ms = 0.f;
                EPR_TRY(cudaEventElapsedTime(&r_ms, e0, e1));
                ms = r_ms < ms ? r_ms : ms;
            }
            if (ms < best) {
                best = ms;
                bTH = t[0];
                bTW = t[1];
                bR = r;
                bO = occ6;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    p->C = saved;
    p->C.smax = bR;
    p->splat_TH = bTH;
    p->splat_TW = bTW;
    p->W.splat_occ6 = bO;
    if (p->has_graph) {
        cudaGraphExecDestroy(p->gexec);
        p->has_graph = false;
    }
    return EPR_OK;
}

// Times the column pass's plans on the spectrum of the solve that just ran
// (each candidate after a fresh forward row pass of the same residual, so
// every timing sees real data): the bulk-copy pass with radix-8 or radix-16
// stages where it exists, and the plain passes with column tiles of 1, 2 and
// 4.  Keeps the fastest and drops the cached graph.  The transforms differ
// only in rounding.
epr_status autotune_col(epr_plan_s* p, const float* D, const float* T, int batch, cudaStream_t s)
{
    const EprConsts& C = p->C;
    const int fwd_mode = 0;
    struct Cand {
        int cw, radix16, occ5;
    };
    const Cand cands[6] = {{0, 0, 0}, {0, 1, 0}, {0, 1, 1}, {1, 0, 0}, {2, 0, 0}, {4, 0, 0}};
    cudaEvent_t e0, e1;
    EPR_TRY(cudaEventCreate(&e0));
    EPR_TRY(cudaEventCreate(&e1));
    float best = 1e30f;
    Cand pick = {p->col_cw, p->W.col_radix16, p->W.col_occ5};
    for (const Cand& c : cands) {
        if (c.radix16 && !(C.ny == 2048 && p->W.col_map)) continue;
        if (p->opt.fft_radix != 0 && c.radix16 != (p->opt.fft_radix == 16)) continue;
        if (c.cw > 0 && C.half % c.cw != 0) continue;
        p->W.col_radix16 = c.radix16;
        p->W.col_occ5 = c.occ5;
        EPR_TRY(cudaMemsetAsync(p->W.st, 0, (size_t)batch * sizeof(EprProjState), s));
        // the column launches alone are timed (the forward row pass before each
        // one only refreshes the spectrum the pass works in place on)
        float ms = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {   // the first repetition warms up; then the fastest
            float r_ms = 0.f;
            for (int k = 0; k < 3; ++k) {
                EPR_TRY(epr_launch_row_fwd(C, p->W, fwd_mode, T, D, nullptr, 0, C.ns, 0, 0.f, batch,
                                           0, s));
                EPR_TRY(cudaEventRecord(e0, s));
                EPR_TRY(epr_launch_col(C, p->W, 0, C.ns, batch, 0, c.cw, -1, s));
                EPR_TRY(cudaEventRecord(e1, s));
                EPR_TRY(cudaEventSynchronize(e1));
                float k_ms = 0.f;
                EPR_TRY(cudaEventElapsedTime(&k_ms, e0, e1));
                r_ms += k_ms;
            }
            if (rep > 0) ms = r_ms < ms ? r_ms : ms;
        }
        if (ms < best) {
            best = ms;
            pick = c;
        }
    }
    p->col_cw = pick.cw;
    p->W.col_radix16 = pick.radix16;
    p->W.col_occ5 = pick.occ5;
    // the one-line 2048-point row passes at five or six blocks per SM: the
    // forward row pass, the chosen column pass and the inverse row pass on a
    // scratch copy of the thickness (the solve's result stays as it is)
    if (C.nx == 2048 && C.ny % 2 == 0 && C.ns == 1) {
        float* Tc = nullptr;
        const size_t n = (size_t)batch * C.nx * C.ny;
        if (cudaMalloc((void**)&Tc, n * sizeof(float)) == cudaSuccess) {
            float best_r = 1e30f;
            int pick_r = p->W.row_occ6;
            for (int occ = 0; occ <= 1; ++occ) {
                p->W.row_occ6 = occ;
                float ms = 1e30f;
                for (int rep = 0; rep < 4; ++rep) {   // a warm-up, then the fastest of three
                    EPR_TRY(cudaMemcpyAsync(Tc, T, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
                    EPR_TRY(cudaEventRecord(e0, s));
                    for (int k = 0; k < 3; ++k) {
                        EPR_TRY(epr_launch_row_fwd(C, p->W, fwd_mode, Tc, D, nullptr, 0, C.ns, 0,
                                                   0.f, batch, 0, s));
                        EPR_TRY(epr_launch_col(C, p->W, 0, C.ns, batch, 0, p->col_cw, -1, s));
                        EPR_TRY(epr_launch_row_inv(C, p->W, 0, Tc, 0, C.ns, 0, 0.4f, 1e-8f, 0.f,
                                                   batch, 0, s));
                    }
                    EPR_TRY(cudaEventRecord(e1, s));
                    EPR_TRY(cudaEventSynchronize(e1));
                    float r_ms = 0.f;
                    EPR_TRY(cudaEventElapsedTime(&r_ms, e0, e1));
                    if (rep > 0) ms = r_ms < ms ? r_ms : ms;
                }
                if (ms < best_r) {
                    best_r = ms;
                    pick_r = occ;
                }
            }
            p->W.row_occ6 = pick_r;
            cudaStreamSynchronize(s);
            cudaFree(Tc);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (p->has_graph) {
        cudaGraphExecDestroy(p->gexec);
        p->has_graph = false;
    }
    return EPR_OK;
}

epr_status solve_common(epr_plan_s* p, const float* D, float* T, int batch, int model,
                        const epr_solve_opts* o, epr_solve_info* info, cudaStream_t s)
{
    if (!p || !D || !T || !o || batch <= 0 || o->n_iter < 0 || !(o->omega > 0.0) || o->tol < 0.0)
        return EPR_ERR_INVALID_ARG;
    if (p->C.xt && model != EPR_MODEL_NONLOCAL) return EPR_ERR_INVALID_ARG;
    if (!aligned16(D) || !aligned16(T)) return EPR_ERR_INVALID_ARG;
    EPR_TRY(cudaSetDevice(p->device));
    const size_t n = (size_t)batch * p->C.nx * p->C.ny;
    epr_status st = ensure_workspace(p, batch, o->n_iter > 0 ? o->n_iter : 1);
    if (st != EPR_OK) return st;
    float *Dd, *Td;
    bool sD, sT;
    // D is the detector image (n / o^2 values with oversampling), T the fine map
    st = resolve(p, 0, D, n / ((size_t)p->C.os * p->C.os), true, s, &Dd, &sD);
    if (st != EPR_OK) return st;
    st = resolve(p, 1, T, n, o->init != 0, s, &Td, &sT);
    if (st != EPR_OK) return st;

    if (p->profiling && o->n_iter > 0) {
        // profiled solve: capture a fresh graph whose kernels are bracketed by
        // event-record nodes, so the kernels run back to back as in the timed
        // solve and the events time the kernels, not the host's launches
        if (p->prof_exec) {
            cudaGraphExecDestroy(p->prof_exec);
            p->prof_exec = nullptr;
        }
        cudaGraph_t g;
        EPR_TRY(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
        const long long before = g_launches.load();
        epr_status ls = launch_solve(p, Dd, Td, batch, o, model, p->cap_stream);
        cudaError_t ce = cudaStreamEndCapture(p->cap_stream, &g);
        const long long captured = g_launches.load() - before;
        g_launches.store(before);
        if (ls != EPR_OK) {
            if (ce == cudaSuccess) cudaGraphDestroy(g);
            return ls;
        }
        EPR_TRY(ce);
        cudaError_t ie = cudaGraphInstantiate(&p->prof_exec, g, 0);
        cudaGraphDestroy(g);
        EPR_TRY(ie);
        EPR_TRY(cudaGraphLaunch(p->prof_exec, s));
        epr_count_launch((int)captured);
    } else if (p->opt.use_graphs && o->n_iter > 0) {
        GraphKey key{Dd, Td, batch, o->n_iter, o->init, model, o->omega, o->tol, o->eps_I};
        if (!(p->has_graph && p->gkey == key)) {
            if (p->has_graph) {
                cudaGraphExecDestroy(p->gexec);
                p->has_graph = false;
            }
            cudaGraph_t g;
            EPR_TRY(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
            const long long before = g_launches.load();
            epr_status ls = launch_solve(p, Dd, Td, batch, o, model, p->cap_stream);
            cudaError_t ce = cudaStreamEndCapture(p->cap_stream, &g);
            const long long captured = g_launches.load() - before;
            g_launches.store(before);  // captured launches did not run
            if (ls != EPR_OK) {
                if (ce == cudaSuccess) cudaGraphDestroy(g);
                return ls;
            }
            EPR_TRY(ce);
            cudaError_t ie = cudaGraphInstantiate(&p->gexec, g, 0);
            cudaGraphDestroy(g);
            EPR_TRY(ie);
            p->gkey = key;
            p->gkernels = (int)captured;
            p->has_graph = true;
        }
        EPR_TRY(cudaGraphLaunch(p->gexec, s));
        epr_count_launch(p->gkernels);
    } else {
        st = launch_solve(p, Dd, Td, batch, o, model, s);
        if (st != EPR_OK) return st;
    }
    if (sT) EPR_TRY(cudaMemcpyAsync(T, Td, n * sizeof(float), cudaMemcpyDeviceToHost, s));

    if (p->opt.autotune && !p->tuned && model == EPR_MODEL_NONLOCAL && o->n_iter > 0) {
        st = autotune_splat(p, Dd, Td, batch, s);
        if (st != EPR_OK) return st;
        // the column pass is timed on the residual of a plain forward (the
        // monochromatic float solve's splat stores it in P; with several
        // lines the split after the last forward of the splat tuner).  Not
        // in fixed-point mode, whose results stay those of the default plan.
        if (p->C.os == 1 && !p->C.xt && !p->C.det) {
            if (p->C.ns > 1) EPR_TRY(epr_launch_split(p->C, p->W, Dd, batch, 0, 0, s));
            st = autotune_col(p, Dd, Td, batch, s);
            if (st != EPR_OK) return st;
        }
    }
    if (info) return collect_info(p, batch, o->n_iter, info, s, 0);
    return EPR_OK;
}

// The per-line constants of a plan from its energies and weights (already
// in p) and L, delta_s, beta_s, derived in double and rounded once to float.
// Returns false when no line is both weighted and absorbing.
bool line_constants(epr_plan_s* p, double L_m, const double* delta, const double* beta)
{
    EprConsts& C = p->C;
    const int n_lines = C.ns, nx = C.nx, ny = C.ny;
    const double pixel_m = p->pixel;
    double wsum = 0.0;
    for (int s = 0; s < n_lines; ++s) wsum += p->w[s];
    double den = 0.0;
    double mu[EPR_MAX_LINES], f[EPR_MAX_LINES];
    EprConsts T = C;   // written back only when valid
    for (int s = 0; s < n_lines; ++s) {
        const double lam = kHcEvM / (p->E[s] * 1e3);
        const double k = 2.0 * kPi / lam;
        mu[s] = 2.0 * k * beta[s];
        f[s] = p->w[s] / wsum;
        den += f[s] * mu[s] * mu[s];
        const double Ld = L_m * delta[s];
        T.f[s] = (float)f[s];
        T.mu[s] = (float)mu[s];
        T.c[s] = (float)(-Ld / (pixel_m * pixel_m));
        const double fx1 = 1.0 / (nx * pixel_m), fy1 = 1.0 / (ny * pixel_m);
        T.ha[s] = mu[s] > 0.0 ? (float)(Ld * 4.0 * kPi * kPi * fx1 * fx1 / mu[s]) : 0.f;
        T.hb[s] = mu[s] > 0.0 ? (float)(Ld * 4.0 * kPi * kPi * fy1 * fy1 / mu[s]) : 0.f;
        const double eps = L_m / k;
        T.qc[s] = (float)(eps * eps / (4.0 * pixel_m * pixel_m * pixel_m * pixel_m));
        T.tneg[s] = mu[s] > 0.0 ? (float)(-0.6931471805599453 / mu[s]) : -3.0e38f;
    }
    if (!(den > 0.0)) return false;
    for (int s = 0; s < n_lines; ++s) T.wproj[s] = (float)(f[s] * mu[s] / den);
    C = T;
    p->L = L_m;
    for (int s = 0; s < n_lines; ++s) {
        p->delta[s] = delta[s];
        p->beta[s] = beta[s];
        p->ha_uniform[s] = C.ha[s];
        p->hb_uniform[s] = C.hb[s];
    }
    return true;
}

std::mutex g_init_mu;
int g_init_done[64];

epr_status init_kernels(int dev)
{
    std::lock_guard<std::mutex> lk(g_init_mu);
    if (dev >= 0 && dev < 64 && g_init_done[dev]) return EPR_OK;
    EPR_TRY(epr_splat_init());
    EPR_TRY(epr_row_init());
    EPR_TRY(epr_col_init());
    EPR_TRY(epr_local_init());
    if (dev >= 0 && dev < 64) g_init_done[dev] = 1;
    return EPR_OK;
}

}  // namespace

// --- C ABI -------------------------------------------------------------------
extern "C" {

const char* epr_status_string(epr_status s)
{
    switch (s) {
    case EPR_OK: return "ok";
    case EPR_ERR_INVALID_ARG: return "invalid argument";
    case EPR_ERR_UNSUPPORTED_SIZE:
        return "unsupported size (need 2^a 3^b, a >= 3, 16..4096; internal grids of an "
               "oversampled plan up to 8192)";
    case EPR_ERR_OOM: return "out of device memory";
    case EPR_ERR_CUDA: return "CUDA error";
    case EPR_ERR_NONFINITE: return "non-finite input";
    case EPR_ERR_TIMEOUT: return "device wait timed out";
    case EPR_ERR_NOT_CONVERGED: return "not converged";
    case EPR_ERR_SHIFT_OVERFLOW: return "overflow list full (shifts beyond max_shift_px)";
    }
    return "unknown status";
}

epr_status epr_plan_create(epr_plan_t* out, int nx, int ny, double pixel_m, double L_m, int n_lines,
                           const double* energy_keV, const double* delta, const double* beta,
                           const double* weights, const epr_options* opt)
{
    if (!out) return EPR_ERR_INVALID_ARG;
    *out = nullptr;
    if (!energy_keV || !delta || !beta || !weights) return EPR_ERR_INVALID_ARG;
    if (n_lines < 1 || n_lines > EPR_MAX_LINES || !(pixel_m > 0.0) || !(L_m >= 0.0))
        return EPR_ERR_INVALID_ARG;
    epr_options o = {4, 0, 0, 1, 0, 0, 0, 0, {0}};
    if (opt) o = *opt;
    if (o.max_shift_px < 1 || o.max_shift_px > EPR_MAX_SHIFT || o.overflow_capacity < 0 ||
        o.oversample < 0 || o.oversample > 16 ||
        !(o.fft_radix == 0 || o.fft_radix == 8 || o.fft_radix == 16))
        return EPR_ERR_INVALID_ARG;
    for (int i = 0; i < 4; ++i)
        if (o.reserved[i] != 0) return EPR_ERR_INVALID_ARG;
    // oversampled internal grid: everything below is the fine grid's
    const int os = o.oversample > 1 ? o.oversample : 1;
    if (nx < 1 || ny < 1 || nx > 4096 || ny > 4096 || nx > 8192 / os || ny > 8192 / os)
        return EPR_ERR_UNSUPPORTED_SIZE;
    nx *= os;
    ny *= os;
    pixel_m /= os;
    if (!size_ok(nx, os > 1 ? 8192 : 4096) || !size_ok(ny, os > 1 ? 8192 : 4096))
        return EPR_ERR_UNSUPPORTED_SIZE;
    double wsum = 0.0;
    for (int s = 0; s < n_lines; ++s) {
        if (!(energy_keV[s] > 0.0) || !(weights[s] >= 0.0) || !(beta[s] >= 0.0) || !isfinite(delta[s]))
            return EPR_ERR_INVALID_ARG;
        wsum += weights[s];
    }
    if (!(wsum > 0.0)) return EPR_ERR_INVALID_ARG;

    epr_plan_s* p = new (std::nothrow) epr_plan_s();
    if (!p) return EPR_ERR_OOM;
    memset(&p->C, 0, sizeof(p->C));
    p->opt = o;
    p->pixel = pixel_m;
    p->L = L_m;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) {
        delete p;
        return EPR_ERR_CUDA;
    }
    EprConsts& C = p->C;
    C.nx = nx;
    C.ny = ny;
    C.ns = n_lines;
    C.half = nx / 2;
    C.smax = o.max_shift_px;
    C.det = o.deterministic ? 1 : 0;
    C.pdl = o.serial_launches ? 0 : 1;
    C.os = os;
    const size_t npix = (size_t)nx * ny;
    C.ovf_cap = o.overflow_capacity > 0 ? o.overflow_capacity
                                        : (int)(npix / 16 > 4096 ? npix / 16 : 4096);
    C.inv_n = (float)(1.0 / ((double)nx * ny));
    for (int s = 0; s < n_lines; ++s) {
        p->E[s] = energy_keV[s];
        p->w[s] = weights[s];
    }
    if (!line_constants(p, L_m, delta, beta)) {
        delete p;
        return EPR_ERR_INVALID_ARG;  // no line both weighted and absorbing
    }

    epr_status st = init_kernels(p->device);
    if (st != EPR_OK) {
        delete p;
        return st;
    }
    // twiddle tables exp(-2 pi i t / n), built in double
    std::vector<float2> tw(nx > ny ? nx : ny);
    for (int t = 0; t < nx; ++t) {
        const double a = -2.0 * kPi * (double)t / nx;
        tw[t] = make_float2((float)cos(a), (float)sin(a));
    }
    e = cudaMalloc((void**)&p->tw_x, nx * sizeof(float2));
    if (e == cudaSuccess) e = cudaMemcpy(p->tw_x, tw.data(), nx * sizeof(float2), cudaMemcpyHostToDevice);
    for (int t = 0; t < ny; ++t) {
        const double a = -2.0 * kPi * (double)t / ny;
        tw[t] = make_float2((float)cos(a), (float)sin(a));
    }
    if (e == cudaSuccess) e = cudaMalloc((void**)&p->tw_y, ny * sizeof(float2));
    if (e == cudaSuccess) e = cudaMemcpy(p->tw_y, tw.data(), ny * sizeof(float2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        if (p->tw_x) cudaFree(p->tw_x);
        if (p->tw_y) cudaFree(p->tw_y);
        delete p;
        return cuda_status(e);
    }
    p->W.tw_x = p->tw_x;
    p->W.tw_y = p->tw_y;
    p->W.col_radix16 = p->opt.fft_radix == 16;   // the choice the tuning calls report
    choose_splat_tiles(p);
    *out = p;
    return EPR_OK;
}

void epr_plan_destroy(epr_plan_t p)
{
    if (!p) return;
    cudaSetDevice(p->device);
    cudaDeviceSynchronize();
    free_workspace(p);
    for (int i = 0; i < 3; ++i)
        if (p->stage[i]) cudaFree(p->stage[i]);
    if (p->tw_x) cudaFree(p->tw_x);
    if (p->tw_y) cudaFree(p->tw_y);
    if (p->h_st) cudaFreeHost(p->h_st);
    if (p->h_hist) cudaFreeHost(p->h_hist);
    if (p->prof_exec) cudaGraphExecDestroy(p->prof_exec);
    if (p->vjp_vx) cudaFree(p->vjp_vx);
    if (p->vjp_vy) cudaFree(p->vjp_vy);
    if (p->vjp_part) cudaFree(p->vjp_part);
    if (p->h_vjp_part) cudaFreeHost(p->h_vjp_part);
    if (p->xt_dev) cudaFree(p->xt_dev);
    for (void* a : p->sv_allocs) cudaFree(a);
    if (p->h_sv_acc) cudaFreeHost(p->h_sv_acc);
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    for (auto& r : p->recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : p->pool) cudaEventDestroy(e);
    delete p;
}

epr_status epr_forward(epr_plan_t p, const float* T, float* P, float* Ps, int batch, int model,
                       void* stream)
{
    if (!p || !T || !P || batch <= 0 || model < 0 || model > 3) return EPR_ERR_INVALID_ARG;
    if (p->C.xt && model != EPR_MODEL_NONLOCAL) return EPR_ERR_INVALID_ARG;
    if (!aligned16(T) || !aligned16(P) || (Ps && !aligned16(Ps))) return EPR_ERR_INVALID_ARG;
    EPR_TRY(cudaSetDevice(p->device));
    cudaStream_t s = (cudaStream_t)stream;
    const EprConsts& C = p->C;
    const size_t npix = (size_t)C.nx * C.ny, n = (size_t)batch * npix;
    epr_status st = ensure_workspace(p, batch, 1);
    if (st != EPR_OK) return st;
    float *Td, *Pd, *Psd = nullptr;
    bool sT, sP, sPs = false;
    // with oversampling P and Ps are detector images: n / o^2 values per map
    const size_t nd = n / ((size_t)C.os * C.os);
    st = resolve(p, 0, T, n, true, s, &Td, &sT);
    if (st == EPR_OK) st = resolve(p, 1, P, nd, false, s, &Pd, &sP);
    if (st == EPR_OK && Ps) st = resolve(p, 2, Ps, nd * C.ns, false, s, &Psd, &sPs);
    if (st != EPR_OK) return st;
    EPR_TRY(cudaMemsetAsync(p->W.st, 0, (size_t)batch * sizeof(EprProjState), s));
    st = launch_forward(p, Td, nullptr, 0, batch, model, 0, s);
    if (st != EPR_OK) return st;
    const bool fx = (model == EPR_MODEL_NONLOCAL) && C.det;
    if (C.os > 1) {
        EPR_TRY(epr_launch_bin_os(C, p->W, fx, Pd, Psd, batch, s));
    } else if (fx) {
        EPR_TRY(epr_launch_fx_to_float(p->W.Pq, Pd, n, s));
        if (Psd) {
            if (C.ns > 1) EPR_TRY(epr_launch_fx_to_float(p->W.Psq, Psd, n * C.ns, s));
            else EPR_TRY(epr_launch_fx_to_float(p->W.Pq, Psd, n, s));
        }
    } else {
        EPR_TRY(cudaMemcpyAsync(Pd, p->W.P, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
        if (Psd) {
            const float* src = C.ns > 1 ? p->W.Ps : p->W.P;
            EPR_TRY(cudaMemcpyAsync(Psd, src, n * C.ns * sizeof(float), cudaMemcpyDeviceToDevice, s));
        }
    }
    if (sP) EPR_TRY(cudaMemcpyAsync(P, Pd, nd * sizeof(float), cudaMemcpyDeviceToHost, s));
    if (sPs) EPR_TRY(cudaMemcpyAsync(Ps, Psd, nd * C.ns * sizeof(float), cudaMemcpyDeviceToHost, s));
    if (sP || sPs) EPR_TRY(cudaStreamSynchronize(s));
    return EPR_OK;
}

epr_status epr_adjoint(epr_plan_t p, const float* T, const float* r, float* g, int line, int batch,
                       void* stream)
{
    if (!p || !T || !r || !g || batch <= 0 || line < 0 || line >= p->C.ns) return EPR_ERR_INVALID_ARG;
    EPR_TRY(cudaSetDevice(p->device));
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = (size_t)batch * p->C.nx * p->C.ny;
    float *Td, *rd, *gd;
    bool sT, sr, sg;
    epr_status st = resolve(p, 0, T, n, true, s, &Td, &sT);
    if (st == EPR_OK) st = resolve(p, 1, r, n, true, s, &rd, &sr);
    if (st == EPR_OK) st = resolve(p, 2, g, n, false, s, &gd, &sg);
    if (st != EPR_OK) return st;
    EPR_TRY(epr_launch_gather(p->C, Td, rd, gd, line, batch, s));
    if (sg) {
        EPR_TRY(cudaMemcpyAsync(g, gd, n * sizeof(float), cudaMemcpyDeviceToHost, s));
        EPR_TRY(cudaStreamSynchronize(s));
    }
    return EPR_OK;
}

epr_status epr_precondition(epr_plan_t p, float* g, int line, int batch, void* stream)
{
    if (!p || !g || batch <= 0 || line < 0 || line >= p->C.ns) return EPR_ERR_INVALID_ARG;
    if (!aligned16(g)) return EPR_ERR_INVALID_ARG;
    // the stand-alone passes run the runtime-sized engine, whose blocks hold
    // rows and columns of up to 4096 points
    if (p->C.nx > 4096 || p->C.ny > 4096) return EPR_ERR_UNSUPPORTED_SIZE;
    EPR_TRY(cudaSetDevice(p->device));
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = (size_t)batch * p->C.nx * p->C.ny;
    epr_status st = ensure_workspace(p, batch, 1);
    if (st != EPR_OK) return st;
    float* gd;
    bool sg;
    st = resolve(p, 0, g, n, true, s, &gd, &sg);
    if (st != EPR_OK) return st;
    EPR_TRY(epr_launch_row_fwd(p->C, p->W, 2, nullptr, nullptr, gd, line, 1, 0, 0.f, batch, 0, s));
    EPR_TRY(epr_launch_col(p->C, p->W, line, 1, batch, 0, 0, -1, s));
    EPR_TRY(epr_launch_row_inv(p->C, p->W, 1, gd, line, 1, 0, 1.f, 0.f, 0.f, batch, 0, s));
    if (sg) {
        EPR_TRY(cudaMemcpyAsync(g, gd, n * sizeof(float), cudaMemcpyDeviceToHost, s));
        EPR_TRY(cudaStreamSynchronize(s));
    }
    return EPR_OK;
}

epr_status epr_solve_nonlocal(epr_plan_t p, const float* D, float* T, int batch,
                              const epr_solve_opts* opts, epr_solve_info* info, void* stream)
{
    return solve_common(p, D, T, batch, EPR_MODEL_NONLOCAL, opts, info, (cudaStream_t)stream);
}

epr_status epr_solve_nonlocal_wkb1(epr_plan_t p, const float* D, float* T, int batch,
                                   const epr_solve_opts* opts, epr_solve_info* info, void* stream)
{
    return solve_common(p, D, T, batch, EPR_MODEL_NONLOCAL_WKB1, opts, info, (cudaStream_t)stream);
}

epr_status epr_solve_local(epr_plan_t p, const float* D, float* T, int batch, int order,
                           const epr_solve_opts* opts, epr_solve_info* info, void* stream)
{
    if (order != 1 && order != 2) return EPR_ERR_INVALID_ARG;
    return solve_common(p, D, T, batch, order, opts, info, (cudaStream_t)stream);
}

epr_status epr_vjp(epr_plan_t p, const float* T, const float* gbar, float* Tbar,
                   double* delta_bar, double* beta_bar, double* L_bar, int batch, void* stream)
{
    if (!p || !T || !gbar || !Tbar || batch <= 0) return EPR_ERR_INVALID_ARG;
    if (p->C.nx < 3 || p->C.ny < 3 || p->C.os > 1 || p->C.xt) return EPR_ERR_INVALID_ARG;
    EPR_TRY(cudaSetDevice(p->device));
    cudaStream_t s = (cudaStream_t)stream;
    const EprConsts& C = p->C;
    const size_t npix = (size_t)C.nx * C.ny, n = (size_t)batch * npix;
    const int nblk = 256;
    if (batch > p->vjp_cap) {
        EPR_TRY(cudaStreamSynchronize(s));
        if (p->vjp_vx) cudaFree(p->vjp_vx);
        if (p->vjp_vy) cudaFree(p->vjp_vy);
        if (p->vjp_part) cudaFree(p->vjp_part);
        if (p->h_vjp_part) cudaFreeHost(p->h_vjp_part);
        p->vjp_vx = p->vjp_vy = nullptr;
        p->vjp_part = p->h_vjp_part = nullptr;
        p->vjp_cap = 0;
        EPR_TRY(cudaMalloc((void**)&p->vjp_vx, n * sizeof(float)));
        EPR_TRY(cudaMalloc((void**)&p->vjp_vy, n * sizeof(float)));
        EPR_TRY(cudaMalloc((void**)&p->vjp_part, (size_t)batch * nblk * 2 * C.ns * sizeof(double)));
        EPR_TRY(cudaMallocHost((void**)&p->h_vjp_part, (size_t)batch * nblk * 2 * C.ns * sizeof(double)));
        p->vjp_cap = batch;
    }
    float *Td, *gd, *Tbd;
    bool sT, sg, sTb;
    epr_status st = resolve(p, 0, T, n, true, s, &Td, &sT);
    if (st == EPR_OK) st = resolve(p, 1, gbar, n, true, s, &gd, &sg);
    if (st == EPR_OK) st = resolve(p, 2, Tbar, n, false, s, &Tbd, &sTb);
    if (st != EPR_OK) return st;
    {
        ProfScope ps(p, EPR_KERNEL_OTHER, s);
        EPR_TRY(epr_launch_vjp(C, Td, gd, Tbd, p->vjp_vx, p->vjp_vy, p->vjp_part, nblk, batch, s));
    }
    if (sTb) EPR_TRY(cudaMemcpyAsync(Tbar, Tbd, n * sizeof(float), cudaMemcpyDeviceToHost, s));
    const bool scalars = delta_bar || beta_bar || L_bar;
    if (scalars) {
        const size_t np = (size_t)batch * nblk * 2 * C.ns;
        EPR_TRY(cudaMemcpyAsync(p->h_vjp_part, p->vjp_part, np * sizeof(double),
                                cudaMemcpyDeviceToHost, s));
    }
    if (scalars || sTb) EPR_TRY(cudaStreamSynchronize(s));
    if (scalars) {
        const double p2 = p->pixel * p->pixel;
        for (int b = 0; b < batch; ++b) {
            double lbar = 0.0;
            for (int l = 0; l < C.ns; ++l) {
                double cbar = 0.0, mubar = 0.0;
                for (int k = 0; k < nblk; ++k) {
                    const double* q = p->h_vjp_part + ((size_t)b * nblk + k) * 2 * C.ns;
                    cbar += q[2 * l];
                    mubar += q[2 * l + 1];
                }
                const double lam = kHcEvM / (p->E[l] * 1e3);
                const double kk = 2.0 * kPi / lam;
                if (delta_bar) delta_bar[(size_t)b * C.ns + l] = -p->L / p2 * cbar;
                if (beta_bar) beta_bar[(size_t)b * C.ns + l] = 2.0 * kk * mubar;
                lbar += -p->delta[l] / p2 * cbar;
            }
            if (L_bar) L_bar[b] = lbar;
        }
    }
    return EPR_OK;
}

}  // extern "C"

// --- reverse mode through the unrolled non-local solve ----------------------
namespace {

// Buffers of the reverse pass for `batch` projections, nck checkpoints and a
// segment of nseg recomputed iterates (allocated once, grown on demand).
epr_status sv_buffers(epr_plan_s* p, int batch, int nck, int nseg)
{
    if (batch <= p->sv_batch && nck <= p->sv_nck && nseg <= p->sv_nseg && p->sv_batch > 0)
        return EPR_OK;
    EPR_TRY(cudaDeviceSynchronize());
    for (void* a : p->sv_allocs) cudaFree(a);
    p->sv_allocs.clear();
    p->sv_batch = p->sv_nck = p->sv_nseg = 0;
    const EprConsts& C = p->C;
    const size_t m = (size_t)batch * C.nx * C.ny, ml = m * C.ns;
    const int nacc = 1 + 3 * C.ns;
    auto get = [&](auto** out, size_t n) -> cudaError_t {
        void* ptr = nullptr;
        cudaError_t e = cudaMalloc(&ptr, n * sizeof(**out) > 0 ? n * sizeof(**out) : 16);
        if (e != cudaSuccess) return e;
        p->sv_allocs.push_back(ptr);
        *out = reinterpret_cast<std::remove_reference_t<decltype(*out)>>(ptr);
        return cudaSuccess;
    };
    cudaError_t e = get(&p->sv_r, m);
    if (e == cudaSuccess) e = get(&p->sv_RS, ml);
    if (e == cudaSuccess) e = get(&p->sv_GA, ml);
    if (e == cudaSuccess) e = get(&p->sv_H, ml);
    if (e == cudaSuccess) e = get(&p->sv_HB, ml);
    if (e == cudaSuccess) e = get(&p->sv_RSB, ml);
    if (e == cudaSuccess) e = get(&p->sv_GB, m);
    if (e == cudaSuccess) e = get(&p->sv_TMP, m);
    if (e == cudaSuccess) e = get(&p->sv_tb, m);
    if (e == cudaSuccess) e = get(&p->sv_tn, m);
    if (e == cudaSuccess) e = get(&p->sv_vx, m);
    if (e == cudaSuccess) e = get(&p->sv_vy, m);
    if (e == cudaSuccess) e = get(&p->sv_Db, m);
    if (e == cudaSuccess) e = get(&p->sv_ck, m * nck);
    if (e == cudaSuccess) e = get(&p->sv_seg, m * (nseg > 0 ? nseg : 1));
    if (e == cudaSuccess) e = get(&p->sv_part, (size_t)batch * epr_sv_blocks() * (C.ns + 1));
    if (e == cudaSuccess) e = get(&p->sv_acc, (size_t)batch * nacc);
    if (e == cudaSuccess) {
        if (p->h_sv_acc) cudaFreeHost(p->h_sv_acc);
        p->h_sv_acc = nullptr;
        e = cudaMallocHost((void**)&p->h_sv_acc, (size_t)batch * nacc * sizeof(double));
    }
    if (e != cudaSuccess) {
        for (void* a : p->sv_allocs) cudaFree(a);
        p->sv_allocs.clear();
        return cuda_status(e);
    }
    p->sv_batch = batch;
    p->sv_nck = nck;
    p->sv_nseg = nseg;
    return EPR_OK;
}

// one iteration of the non-local solve in place on T (batch projections)
epr_status sv_step(epr_plan_s* p, const float* D, float* T, int batch, double omega, double eps,
                   cudaStream_t s)
{
    epr_solve_opts o1 = {1, omega, 0.0, eps, 1};
    return launch_solve(p, D, T, batch, &o1, EPR_MODEL_NONLOCAL, s);
}

// the preconditioner of line s in place on a batch of maps, or with symbol
// kind 1 / 2 (dH/dmu, dH/d(L delta)) of the generic column pass
epr_status sv_filter(epr_plan_s* p, float* g, int s, int kind, float kscale, int batch,
                     cudaStream_t st)
{
    const EprConsts& C = p->C;
    EPR_TRY(epr_launch_row_fwd(C, p->W, 2, nullptr, nullptr, g, s, 1, 0, 0.f, batch, 0, st));
    if (kind == 0) EPR_TRY(epr_launch_col(C, p->W, s, 1, batch, 0, 0, -1, st));
    else EPR_TRY(epr_launch_col_kind(C, p->W, s, batch, kind, kscale, st));
    EPR_TRY(epr_launch_row_inv(C, p->W, 1, g, s, 1, 0, 1.f, 0.f, 0.f, batch, 0, st));
    return EPR_OK;
}

// The reverse of one iteration at thickness T: tb (dF/dT') -> tn (dF/dT),
// Db += dF/dD, scalar accumulators += their shares.
epr_status sv_reverse_iteration(epr_plan_s* p, const float* D, const float* T, int B, double omega,
                                double eps, cudaStream_t st)
{
    const EprConsts& C = p->C;
    const int ns = C.ns, nacc = 1 + 3 * ns;
    const size_t npix = (size_t)C.nx * C.ny, m = (size_t)B * npix;
    // forward of this iteration, recomputed: P, P_s (float), r, r_s, g_s, h_s
    EPR_TRY(cudaMemsetAsync(p->W.st, 0, (size_t)B * sizeof(EprProjState), st));
    epr_status es = launch_forward(p, T, nullptr, 0, B, EPR_MODEL_NONLOCAL, 0, st);
    if (es != EPR_OK) return es;
    if (C.det) {
        EPR_TRY(epr_launch_fx_to_float(p->W.Pq, p->W.P, m, st));
        if (ns > 1) EPR_TRY(epr_launch_fx_to_float(p->W.Psq, p->W.Ps, m * ns, st));
    }
    EPR_TRY(epr_launch_sv_split(C, D, p->W.P, p->W.Ps, p->sv_r, p->sv_RS, B, st));
    for (int s = 0; s < ns; ++s) {
        EPR_TRY(epr_launch_gather(C, T, p->sv_RS + s * m, p->sv_GA + s * m, s, B, st));
        EPR_TRY(cudaMemcpyAsync(p->sv_H + s * m, p->sv_GA + s * m, m * sizeof(float),
                                cudaMemcpyDeviceToDevice, st));
        es = sv_filter(p, p->sv_H + s * m, s, 0, 0.f, B, st);
        if (es != EPR_OK) return es;
    }
    // reverse
    EPR_TRY(cudaMemsetAsync(p->sv_tn, 0, m * sizeof(float), st));
    EPR_TRY(cudaMemsetAsync(p->sv_vx, 0, m * sizeof(float), st));
    EPR_TRY(cudaMemsetAsync(p->sv_vy, 0, m * sizeof(float), st));
    EPR_TRY(cudaMemsetAsync(p->sv_RSB, 0, m * ns * sizeof(float), st));
    double den = 0.0;
    for (int s = 0; s < ns; ++s) den += (double)C.f[s] * C.mu[s] * C.mu[s];
    EPR_TRY(epr_launch_sv_update_adj(C, T, p->sv_H, p->sv_tb, p->sv_HB, p->sv_part, B,
                                     (float)omega, (float)eps, (float)(1.0 / den), st));
    EPR_TRY(epr_launch_sv_accum(p->sv_part, npix, ns + 1, 0, p->sv_acc, nacc, 0, 1.0, B, st));
    for (int s = 0; s < ns; ++s)
        EPR_TRY(epr_launch_sv_accum(p->sv_part, npix, ns + 1, 1 + s, p->sv_acc, nacc, 1 + s, 1.0, B, st));
    for (int s = 0; s < ns; ++s) {
        float* HBs = p->sv_HB + s * m;
        // gbar_s = H_s hbar_s
        EPR_TRY(cudaMemcpyAsync(p->sv_GB, HBs, m * sizeof(float), cudaMemcpyDeviceToDevice, st));
        es = sv_filter(p, p->sv_GB, s, 0, 0.f, B, st);
        if (es != EPR_OK) return es;
        // the symbol's dependence on mu_s and L delta_s: <hbar_s, dH g_s>
        const double Ld = p->L * p->delta[s];
        for (int kind = 1; kind <= 2; ++kind) {
            EPR_TRY(cudaMemcpyAsync(p->sv_TMP, p->sv_GA + s * m, m * sizeof(float),
                                    cudaMemcpyDeviceToDevice, st));
            const float ks = kind == 1 ? (float)(1.0 / C.mu[s]) : (float)(-1.0 / Ld);
            es = sv_filter(p, p->sv_TMP, s, kind, ks, B, st);
            if (es != EPR_OK) return es;
            EPR_TRY(epr_launch_sv_dot(HBs, p->sv_TMP, npix, p->sv_part, B, st));
            EPR_TRY(epr_launch_sv_accum(p->sv_part, npix, 1, 0, p->sv_acc, nacc,
                                        kind == 1 ? 1 + s : 1 + ns + s, 1.0, B, st));
        }
        // the gather backwards: input adjoint (a splat) and shift term
        EPR_TRY(epr_launch_sv_splat_field(C, T, p->sv_GB, p->sv_RSB + s * m, s, B, st));
        EPR_TRY(epr_launch_sv_interp_du(C, 0, T, p->sv_RS + s * m, p->sv_GB, nullptr, p->sv_vx,
                                        p->sv_vy, p->sv_tn, p->sv_part, s, (float)omega, B, st));
        EPR_TRY(epr_launch_sv_accum(p->sv_part, npix, 2, 0, p->sv_acc, nacc, 1 + 2 * ns + s, 1.0, B, st));
    }
    // the split, then the splat backwards (input and shift) with I_s's share
    EPR_TRY(epr_launch_sv_split_adj(C, p->sv_RSB, p->W.P, p->W.Ps, p->sv_r, p->sv_Db, B, st));
    for (int s = 0; s < ns; ++s) {
        EPR_TRY(epr_launch_sv_interp_du(C, 1, T, p->sv_RSB + s * m, nullptr, p->sv_HB + s * m,
                                        p->sv_vx, p->sv_vy, p->sv_tn, p->sv_part, s, (float)omega,
                                        B, st));
        EPR_TRY(epr_launch_sv_accum(p->sv_part, npix, 2, 0, p->sv_acc, nacc, 1 + 2 * ns + s, 1.0, B, st));
        EPR_TRY(epr_launch_sv_accum(p->sv_part, npix, 2, 1, p->sv_acc, nacc, 1 + s, 1.0, B, st));
    }
    EPR_TRY(epr_launch_sv_gT(C, p->sv_vx, p->sv_vy, p->sv_tn, B, st));
    std::swap(p->sv_tb, p->sv_tn);
    return EPR_OK;
}

}  // namespace

extern "C" {

epr_status epr_solve_vjp(epr_plan_t p, const float* D, const float* T0, int batch, int n_iter,
                         double omega, double eps_I, int checkpoint_every, const float* Tbar,
                         float* T_out, float* T0_bar, float* D_bar, double* delta_bar,
                         double* beta_bar, double* L_bar, void* stream)
{
    if (!p || !D || !Tbar || batch <= 0 || n_iter < 0 || !(omega > 0.0) || checkpoint_every < 0)
        return EPR_ERR_INVALID_ARG;
    const EprConsts& C = p->C;
    if (C.os > 1 || C.xt) return EPR_ERR_INVALID_ARG;
    for (int s = 0; s < C.ns; ++s)
        if (!(C.mu[s] > 0.f) || !(p->L * p->delta[s] > 0.0)) return EPR_ERR_INVALID_ARG;
    const float* dev_in[3] = {D, T0, Tbar};
    float* dev_out[3] = {T_out, T0_bar, D_bar};
    for (const float* a : dev_in)
        if (a && (!is_device_ptr(a) || !aligned16(a))) return EPR_ERR_INVALID_ARG;
    for (float* a : dev_out)
        if (a && (!is_device_ptr(a) || !aligned16(a))) return EPR_ERR_INVALID_ARG;
    EPR_TRY(cudaSetDevice(p->device));
    cudaStream_t st = (cudaStream_t)stream;
    const double eps = eps_I > 0 ? eps_I : 1e-8;
    const int mck = checkpoint_every > 0 ? checkpoint_every : 1;   // iterations per checkpoint
    const int nck = n_iter / mck + 1;
    epr_status es = ensure_workspace(p, batch, 1);
    if (es != EPR_OK) return es;
    es = sv_buffers(p, batch, nck, mck > 1 ? mck : 0);
    if (es != EPR_OK) return es;
    const size_t m = (size_t)batch * C.nx * C.ny;
    const int nacc = 1 + 3 * C.ns;
    // forward: the iterates tau_0, tau_mck, tau_2 mck, ... kept; tau_N in sv_tn
    float* Tc = p->sv_tn;
    if (T0) EPR_TRY(cudaMemcpyAsync(Tc, T0, m * sizeof(float), cudaMemcpyDeviceToDevice, st));
    else EPR_TRY(cudaMemsetAsync(Tc, 0, m * sizeof(float), st));
    for (int it = 0; it < n_iter; ++it) {
        if (it % mck == 0)
            EPR_TRY(cudaMemcpyAsync(p->sv_ck + (size_t)(it / mck) * m, Tc, m * sizeof(float),
                                    cudaMemcpyDeviceToDevice, st));
        es = sv_step(p, D, Tc, batch, omega, eps, st);
        if (es != EPR_OK) return es;
    }
    if (T_out) EPR_TRY(cudaMemcpyAsync(T_out, Tc, m * sizeof(float), cudaMemcpyDeviceToDevice, st));
    // reverse, segment by segment from the last
    EPR_TRY(cudaMemcpyAsync(p->sv_tb, Tbar, m * sizeof(float), cudaMemcpyDeviceToDevice, st));
    EPR_TRY(cudaMemsetAsync(p->sv_Db, 0, m * sizeof(float), st));
    EPR_TRY(cudaMemsetAsync(p->sv_acc, 0, (size_t)batch * nacc * sizeof(double), st));
    for (int seg = (n_iter - 1) / mck; n_iter > 0 && seg >= 0; --seg) {
        const int base = seg * mck, len = (n_iter - base) < mck ? (n_iter - base) : mck;
        const float* ck = p->sv_ck + (size_t)seg * m;
        if (mck > 1) {   // recompute the segment's iterates from its checkpoint
            EPR_TRY(cudaMemcpyAsync(p->sv_seg, ck, m * sizeof(float), cudaMemcpyDeviceToDevice, st));
            for (int i = 1; i < len; ++i) {
                float* Ti = p->sv_seg + (size_t)i * m;
                EPR_TRY(cudaMemcpyAsync(Ti, Ti - m, m * sizeof(float), cudaMemcpyDeviceToDevice, st));
                es = sv_step(p, D, Ti, batch, omega, eps, st);
                if (es != EPR_OK) return es;
            }
        }
        for (int i = len - 1; i >= 0; --i) {
            const float* Ti = mck > 1 ? p->sv_seg + (size_t)i * m : ck;
            es = sv_reverse_iteration(p, D, Ti, batch, omega, eps, st);
            if (es != EPR_OK) return es;
        }
    }
    if (T0_bar) EPR_TRY(cudaMemcpyAsync(T0_bar, p->sv_tb, m * sizeof(float), cudaMemcpyDeviceToDevice, st));
    if (D_bar) EPR_TRY(cudaMemcpyAsync(D_bar, p->sv_Db, m * sizeof(float), cudaMemcpyDeviceToDevice, st));
    const bool scalars = delta_bar || beta_bar || L_bar;
    if (scalars) {
        EPR_TRY(cudaMemcpyAsync(p->h_sv_acc, p->sv_acc, (size_t)batch * nacc * sizeof(double),
                                cudaMemcpyDeviceToHost, st));
        EPR_TRY(cudaStreamSynchronize(st));
        // back from c_s = -L delta_s / p^2, the filter's L delta_s and mu_s = 2 k_s beta_s
        const double p2 = p->pixel * p->pixel;
        double wsum = 0.0;
        for (int s = 0; s < C.ns; ++s) wsum += p->w[s];
        for (int b = 0; b < batch; ++b) {
            const double* a = p->h_sv_acc + (size_t)b * nacc;
            double lbar = 0.0;
            for (int s = 0; s < C.ns; ++s) {
                const double lam = kHcEvM / (p->E[s] * 1e3);
                const double k = 2.0 * kPi / lam;
                const double mu = 2.0 * k * p->beta[s], f = p->w[s] / wsum;
                const double mub = a[1 + s] + a[0] * 2.0 * f * mu;
                const double Ldb = a[1 + C.ns + s], cb = a[1 + 2 * C.ns + s];
                if (delta_bar) delta_bar[(size_t)b * C.ns + s] = -p->L / p2 * cb + p->L * Ldb;
                if (beta_bar) beta_bar[(size_t)b * C.ns + s] = 2.0 * k * mub;
                lbar += -p->delta[s] / p2 * cb + p->delta[s] * Ldb;
            }
            if (L_bar) L_bar[b] = lbar;
        }
    }
    return EPR_OK;
}

epr_status epr_plan_set_params(epr_plan_t p, double L_m, const double* delta, const double* beta)
{
    if (!p || !delta || !beta || !(L_m >= 0.0) || !isfinite(L_m) || p->C.xt)
        return EPR_ERR_INVALID_ARG;
    for (int s = 0; s < p->C.ns; ++s)
        if (!(beta[s] >= 0.0) || !isfinite(beta[s]) || !isfinite(delta[s])) return EPR_ERR_INVALID_ARG;
    EPR_TRY(cudaSetDevice(p->device));
    // graphs and work in flight hold the old constants by value; nothing is
    // reallocated, so letting queued work finish first is enough
    if (!line_constants(p, L_m, delta, beta)) return EPR_ERR_INVALID_ARG;
    if (p->has_graph) {
        cudaGraphExecDestroy(p->gexec);
        p->has_graph = false;
    }
    if (p->prof_exec) {
        cudaGraphExecDestroy(p->prof_exec);
        p->prof_exec = nullptr;
    }
    return EPR_OK;
}

epr_status epr_plan_set_xspec(epr_plan_t p, const epr_xspec* tab)
{
    if (!p) return EPR_ERR_INVALID_ARG;
    EPR_TRY(cudaSetDevice(p->device));
    EprConsts& C = p->C;
    const int ns = C.ns, nx = C.nx;
    if (!tab) {   // back to the uniform spectrum of the plan
        EPR_TRY(cudaDeviceSynchronize());
        if (p->xt_dev) cudaFree(p->xt_dev);
        p->xt_dev = nullptr;
        C.xt = nullptr;
        for (int s = 0; s < ns; ++s) {
            C.ha[s] = p->ha_uniform[s];
            C.hb[s] = p->hb_uniform[s];
        }
    } else {
        const int K = tab->n_knots;
        if (K < 1 || !tab->x_knots || !tab->weights || !tab->delta || !tab->beta || C.os > 1)
            return EPR_ERR_INVALID_ARG;
        for (int k = 0; k < K; ++k)
            if (!isfinite(tab->x_knots[k]) || (k > 0 && !(tab->x_knots[k] > tab->x_knots[k - 1])))
                return EPR_ERR_INVALID_ARG;
        for (int i = 0; i < ns * K; ++i)
            if (!(tab->weights[i] > 0.0) || !isfinite(tab->weights[i]) || !(tab->beta[i] >= 0.0) ||
                !isfinite(tab->beta[i]) || !isfinite(tab->delta[i]))
                return EPR_ERR_INVALID_ARG;
        // each knot value at column x: linear between the knots around x,
        // constant beyond the first and the last
        auto at = [&](const double* v, double x) {
            const double* X = tab->x_knots;
            if (x <= X[0]) return v[0];
            if (x >= X[K - 1]) return v[K - 1];
            int k = 1;
            while (X[k] < x) ++k;   // X[k - 1] < x <= X[k]
            const double t = (x - X[k - 1]) / (X[k] - X[k - 1]);
            return v[k - 1] + t * (v[k] - v[k - 1]);
        };
        const double kPi = 3.14159265358979323846;
        std::vector<float> h((size_t)EPR_XT_KINDS * ns * nx);
        std::vector<double> f(ns), mu(ns), dl(ns), mu_mean(ns, 0.0), ld_mean(ns, 0.0);
        auto put = [&](int kind, int s, int x, double v) {
            h[((size_t)kind * ns + s) * nx + x] = (float)v;
        };
        for (int x = 0; x < nx; ++x) {
            double wsum = 0.0, den = 0.0;
            for (int s = 0; s < ns; ++s) {
                f[s] = at(tab->weights + (size_t)s * K, (double)x);
                wsum += f[s];
            }
            for (int s = 0; s < ns; ++s) {
                const double lam = kHcEvM / (p->E[s] * 1e3);
                const double k = 2.0 * kPi / lam;
                f[s] /= wsum;
                mu[s] = 2.0 * k * at(tab->beta + (size_t)s * K, (double)x);
                dl[s] = at(tab->delta + (size_t)s * K, (double)x);
                den += f[s] * mu[s] * mu[s];
                mu_mean[s] += mu[s] / nx;
                ld_mean[s] += p->L * dl[s] / nx;
            }
            if (!(den > 0.0)) return EPR_ERR_INVALID_ARG;   // no absorbing line in column x
            for (int s = 0; s < ns; ++s) {
                put(EPR_XT_F, s, x, f[s]);
                put(EPR_XT_MU, s, x, mu[s]);
                put(EPR_XT_C, s, x, -p->L * dl[s] / (p->pixel * p->pixel));
                put(EPR_XT_WPROJ, s, x, f[s] * mu[s] / den);
                put(EPR_XT_TNEG, s, x, mu[s] > 0.0 ? -0.6931471805599453 / mu[s] : -3.0e38);
            }
        }
        EPR_TRY(cudaDeviceSynchronize());
        if (!p->xt_dev) EPR_TRY(cudaMalloc((void**)&p->xt_dev, h.size() * sizeof(float)));
        EPR_TRY(cudaMemcpy(p->xt_dev, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice));
        C.xt = p->xt_dev;
        // the preconditioner must be FFT-diagonal: each line's column means
        const double fx1 = 1.0 / (nx * p->pixel), fy1 = 1.0 / (C.ny * p->pixel);
        for (int s = 0; s < ns; ++s) {
            C.ha[s] = mu_mean[s] > 0.0 ? (float)(ld_mean[s] * 4.0 * kPi * kPi * fx1 * fx1 / mu_mean[s]) : 0.f;
            C.hb[s] = mu_mean[s] > 0.0 ? (float)(ld_mean[s] * 4.0 * kPi * kPi * fy1 * fy1 / mu_mean[s]) : 0.f;
        }
    }
    // kernels take the constants by value: cached graphs are stale
    if (p->has_graph) {
        cudaGraphExecDestroy(p->gexec);
        p->has_graph = false;
    }
    if (p->prof_exec) {
        cudaGraphExecDestroy(p->prof_exec);
        p->prof_exec = nullptr;
    }
    return EPR_OK;
}

epr_status epr_plan_get_tuning(epr_plan_t p, int* out)
{
    if (!p || !out) return EPR_ERR_INVALID_ARG;
    out[0] = p->splat_TH;
    out[1] = p->splat_TW;
    out[2] = p->C.smax;
    out[3] = p->col_cw;
    out[4] = p->W.col_radix16 ? 16 : 8;
    out[5] = p->W.row_occ6 ? 6 : 5;
    out[6] = p->W.col_occ5 ? 5 : 4;
    out[7] = p->W.splat_occ6 ? 6 : 5;
    out[8] = p->tuned ? 1 : 0;
    return EPR_OK;
}

epr_status epr_plan_set_tuning(epr_plan_t p, const int* in)
{
    if (!p || !in) return EPR_ERR_INVALID_ARG;
    const int th = in[0], tw = in[1], reach = in[2], cw = in[3], radix = in[4], occ = in[5];
    const int cocc = in[6], socc = in[7];
    const bool tile_ok = (th == 64 || th == 32) && (tw == 64 || tw == 32);
    if (!tile_ok || reach < 1 || reach > EPR_MAX_SHIFT || !(cw == 0 || cw == 1 || cw == 2 || cw == 4) ||
        !(radix == 8 || radix == 16) || !(occ == 5 || occ == 6) || !(cocc == 4 || cocc == 5) ||
        (cocc == 5 && radix != 16) || !(socc == 5 || socc == 6) ||
        (socc == 6 && !epr_splat_has_occ6(th, tw, reach)))
        return EPR_ERR_INVALID_ARG;
    EprConsts C = p->C;
    C.smax = reach;
    if ((size_t)C.ns * th * tw * (C.det ? 8 : 4) > 65536) return EPR_ERR_INVALID_ARG;
    int optin = 0;
    EPR_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device));
    if (epr_splat_smem(C, th, tw) + 4096 > (size_t)optin) return EPR_ERR_INVALID_ARG;
    p->C.smax = reach;
    p->splat_TH = th;
    p->splat_TW = tw;
    p->col_cw = cw;
    p->W.col_radix16 = radix == 16;
    p->W.row_occ6 = occ == 6;
    p->W.col_occ5 = cocc == 5;
    p->W.splat_occ6 = socc == 6;
    p->tuned = true;   // the autotuner does not run over an explicit choice
    if (p->has_graph) {
        cudaGraphExecDestroy(p->gexec);
        p->has_graph = false;
    }
    return EPR_OK;
}

epr_status epr_check_device_status(epr_plan_t p, void* stream)
{
    if (!p) return EPR_ERR_INVALID_ARG;
    if (!p->W.err) return EPR_OK;
    EPR_TRY(cudaSetDevice(p->device));
    cudaStream_t s = (cudaStream_t)stream;
    unsigned int herr = 0;
    EPR_TRY(cudaMemcpyAsync(&herr, p->W.err, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
    EPR_TRY(cudaMemsetAsync(p->W.err, 0, sizeof(unsigned int), s));
    EPR_TRY(cudaStreamSynchronize(s));
    if (herr & EPR_DEVERR_NONFINITE) return EPR_ERR_NONFINITE;
    if (herr & EPR_DEVERR_TIMEOUT) return EPR_ERR_TIMEOUT;
    if (herr & EPR_DEVERR_OVERFLOW) return EPR_ERR_SHIFT_OVERFLOW;
    return EPR_OK;
}

epr_status epr_profile_enable(epr_plan_t p, int enable)
{
    if (!p) return EPR_ERR_INVALID_ARG;
    EPR_TRY(cudaSetDevice(p->device));
    if (!enable) {
        EPR_TRY(cudaDeviceSynchronize());
        for (auto& r : p->recs) {
            p->pool.push_back(r.a);
            p->pool.push_back(r.b);
        }
        p->recs.clear();
    }
    if (enable) {
        while (p->pool.size() + 2 * p->recs.size() < (size_t)kProfEvents) {
            cudaEvent_t e = nullptr;
            EPR_TRY(cudaEventCreate(&e));
            p->pool.push_back(e);
        }
    }
    p->profiling = enable != 0;
    return EPR_OK;
}

epr_status epr_profile_read(epr_plan_t p, int* launches, double* total_ms)
{
    if (!p || !launches || !total_ms) return EPR_ERR_INVALID_ARG;
    EPR_TRY(cudaSetDevice(p->device));
    for (int k = 0; k < EPR_KERNEL_KINDS; ++k) {
        launches[k] = 0;
        total_ms[k] = 0.0;
    }
    for (auto& r : p->recs) {
        EPR_TRY(cudaEventSynchronize(r.b));
        float ms = 0.f;
        EPR_TRY(cudaEventElapsedTime(&ms, r.a, r.b));
        if (r.kind >= 0 && r.kind < EPR_KERNEL_KINDS) {
            launches[r.kind] += 1;
            total_ms[r.kind] += ms;
        }
        p->pool.push_back(r.a);
        p->pool.push_back(r.b);
    }
    p->recs.clear();
    return EPR_OK;
}

}  // extern "C"

// --- batched solve of uneven sizes ----------------------------------------------
struct epr_batch_s {
    double pixel, L;
    int ns;
    double E[EPR_MAX_LINES], delta[EPR_MAX_LINES], beta[EPR_MAX_LINES], w[EPR_MAX_LINES];
    epr_options opt;
    int device;
    struct Group {
        int nx, ny;
        epr_plan_t plan;
        float* D;       // gathered data [cap][ny][nx]
        float* T;       // gathered thickness
        int cap;
        cudaStream_t stream;
        cudaEvent_t done;
    };
    std::vector<Group> groups;
    cudaEvent_t start;
};

namespace {

// Index of the group for size nx x ny with room for `count` projections
// (created or grown on demand), or -1 with *st set.
int batch_group(epr_batch_s* bp, int nx, int ny, int count, epr_status* st)
{
    *st = EPR_OK;
    for (size_t gi = 0; gi < bp->groups.size(); ++gi) {
        epr_batch_s::Group& g = bp->groups[gi];
        if (g.nx == nx && g.ny == ny) {
            if (g.cap < count) {
                cudaStreamSynchronize(g.stream);
                cudaFree(g.D);
                cudaFree(g.T);
                g.D = g.T = nullptr;
                g.cap = 0;
                const size_t n = (size_t)count * nx * ny;
                if (cudaMalloc((void**)&g.D, n * sizeof(float)) != cudaSuccess ||
                    cudaMalloc((void**)&g.T, n * sizeof(float)) != cudaSuccess) {
                    *st = EPR_ERR_OOM;
                    return -1;
                }
                g.cap = count;
            }
            return (int)gi;
        }
    }
    epr_batch_s::Group g = {};
    g.nx = nx;
    g.ny = ny;
    *st = epr_plan_create(&g.plan, nx, ny, bp->pixel, bp->L, bp->ns, bp->E, bp->delta, bp->beta,
                          bp->w, &bp->opt);
    if (*st != EPR_OK) return -1;
    const size_t n = (size_t)count * nx * ny;
    if (cudaMalloc((void**)&g.D, n * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void**)&g.T, n * sizeof(float)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming) != cudaSuccess) {
        *st = EPR_ERR_OOM;
        if (g.D) cudaFree(g.D);
        if (g.T) cudaFree(g.T);
        epr_plan_destroy(g.plan);
        return -1;
    }
    g.cap = count;
    bp->groups.push_back(g);
    return (int)bp->groups.size() - 1;
}

}  // namespace

extern "C" {

epr_status epr_batch_create(epr_batch_t* out, double pixel_m, double L_m, int n_lines,
                            const double* energy_keV, const double* delta, const double* beta,
                            const double* weights, const epr_options* opt)
{
    if (!out) return EPR_ERR_INVALID_ARG;
    *out = nullptr;
    if (!energy_keV || !delta || !beta || !weights || n_lines < 1 || n_lines > EPR_MAX_LINES ||
        !(pixel_m > 0.0) || !(L_m >= 0.0))
        return EPR_ERR_INVALID_ARG;
    epr_batch_s* bp = new (std::nothrow) epr_batch_s();
    if (!bp) return EPR_ERR_OOM;
    bp->pixel = pixel_m;
    bp->L = L_m;
    bp->ns = n_lines;
    for (int s = 0; s < n_lines; ++s) {
        bp->E[s] = energy_keV[s];
        bp->delta[s] = delta[s];
        bp->beta[s] = beta[s];
        bp->w[s] = weights[s];
    }
    epr_options o = {4, 0, 0, 1, 0, 0, 0, 0, {0}};
    if (opt) o = *opt;
    if (o.oversample > 1) {   // detector and internal sizes differ: plans only
        delete bp;
        return EPR_ERR_INVALID_ARG;
    }
    bp->opt = o;
    if (cudaGetDevice(&bp->device) != cudaSuccess ||
        cudaEventCreateWithFlags(&bp->start, cudaEventDisableTiming) != cudaSuccess) {
        delete bp;
        return EPR_ERR_CUDA;
    }
    *out = bp;
    return EPR_OK;
}

void epr_batch_destroy(epr_batch_t bp)
{
    if (!bp) return;
    cudaSetDevice(bp->device);
    cudaDeviceSynchronize();
    for (auto& g : bp->groups) {
        epr_plan_destroy(g.plan);
        cudaFree(g.D);
        cudaFree(g.T);
        cudaStreamDestroy(g.stream);
        cudaEventDestroy(g.done);
    }
    cudaEventDestroy(bp->start);
    delete bp;
}

epr_status epr_solve_nonlocal_batched(epr_batch_t bp, const epr_batch_desc* descs, int n,
                                      const epr_solve_opts* opts, epr_solve_info* info,
                                      void* stream)
{
    if (!bp || !descs || n <= 0 || !opts) return EPR_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i) {
        if (!descs[i].D || !descs[i].T) return EPR_ERR_INVALID_ARG;
        if (!size_ok(descs[i].nx) || !size_ok(descs[i].ny)) return EPR_ERR_UNSUPPORTED_SIZE;
    }
    EPR_TRY(cudaSetDevice(bp->device));
    cudaStream_t s = (cudaStream_t)stream;
    // size groups, in order of first appearance
    std::vector<std::pair<int, int>> sizes;
    std::vector<std::vector<int>> members;
    for (int i = 0; i < n; ++i) {
        size_t k = 0;
        while (k < sizes.size() && !(sizes[k].first == descs[i].nx && sizes[k].second == descs[i].ny)) ++k;
        if (k == sizes.size()) {
            sizes.push_back({descs[i].nx, descs[i].ny});
            members.emplace_back();
        }
        members[k].push_back(i);
    }
    EPR_TRY(cudaEventRecord(bp->start, s));
    std::vector<int> used;
    for (size_t k = 0; k < sizes.size(); ++k) {
        const int cnt = (int)members[k].size();
        epr_status st;
        const int gi = batch_group(bp, sizes[k].first, sizes[k].second, cnt, &st);
        if (gi < 0) return st;
        used.push_back(gi);
        epr_batch_s::Group* g = &bp->groups[gi];
        const size_t npix = (size_t)g->nx * g->ny;
        EPR_TRY(cudaStreamWaitEvent(g->stream, bp->start, 0));
        for (int j = 0; j < cnt; ++j) {
            const epr_batch_desc& d = descs[members[k][j]];
            EPR_TRY(cudaMemcpyAsync(g->D + j * npix, d.D, npix * sizeof(float), cudaMemcpyDefault,
                                    g->stream));
            if (opts->init)
                EPR_TRY(cudaMemcpyAsync(g->T + j * npix, d.T, npix * sizeof(float),
                                        cudaMemcpyDefault, g->stream));
        }
        st = solve_common(g->plan, g->D, g->T, cnt, EPR_MODEL_NONLOCAL, opts, nullptr, g->stream);
        if (st != EPR_OK) return st;
        for (int j = 0; j < cnt; ++j) {
            const epr_batch_desc& d = descs[members[k][j]];
            EPR_TRY(cudaMemcpyAsync(d.T, g->T + j * npix, npix * sizeof(float), cudaMemcpyDefault,
                                    g->stream));
        }
        EPR_TRY(cudaEventRecord(g->done, g->stream));
        EPR_TRY(cudaStreamWaitEvent(s, g->done, 0));
    }
    if (info) {
        // per-projection results in the order of descs
        epr_solve_info part = *info;
        std::vector<int> it_tmp;
        std::vector<double> r_tmp, k_tmp, rh_tmp, kh_tmp;
        epr_status worst = EPR_OK;
        info->overflow_sources = 0;
        for (size_t k = 0; k < sizes.size(); ++k) {
            const int cnt = (int)members[k].size();
            const int nh = opts->n_iter > 0 ? opts->n_iter : 1;
            it_tmp.assign(cnt, 0);
            r_tmp.assign(cnt, 0.0);
            k_tmp.assign(cnt, 0.0);
            rh_tmp.assign((size_t)cnt * nh, 0.0);
            kh_tmp.assign((size_t)cnt * nh, 0.0);
            part.iters = it_tmp.data();
            part.rho = r_tmp.data();
            part.kappa = k_tmp.data();
            part.rho_hist = rh_tmp.data();
            part.kappa_hist = kh_tmp.data();
            part.overflow_sources = 0;
            const epr_batch_s::Group& g = bp->groups[used[k]];
            epr_status st = collect_info(g.plan, cnt, opts->n_iter, &part, g.stream, 0);
            if (st != EPR_OK) worst = st;
            for (int j = 0; j < cnt; ++j) {
                const int i = members[k][j];
                if (info->iters) info->iters[i] = it_tmp[j];
                if (info->rho) info->rho[i] = r_tmp[j];
                if (info->kappa) info->kappa[i] = k_tmp[j];
                for (int q = 0; q < opts->n_iter; ++q) {
                    if (info->rho_hist) info->rho_hist[(size_t)i * opts->n_iter + q] = rh_tmp[(size_t)j * opts->n_iter + q];
                    if (info->kappa_hist) info->kappa_hist[(size_t)i * opts->n_iter + q] = kh_tmp[(size_t)j * opts->n_iter + q];
                }
            }
            info->overflow_sources += part.overflow_sources;
        }
        EPR_TRY(cudaStreamSynchronize(s));
        return worst;
    }
    return EPR_OK;
}

}  // extern "C"

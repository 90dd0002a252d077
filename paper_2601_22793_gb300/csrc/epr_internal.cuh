// Internal definitions shared by the CUDA translation units of libepr.
// Nothing here is part of the C ABI (include/epr.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "epr.h"

#define EPR_MAX_LINES 16
#define EPR_MAX_SHIFT 32

// Device-side error bits (OR-ed into the plan's error word).
#define EPR_DEVERR_OVERFLOW 1u
#define EPR_DEVERR_TIMEOUT 2u    // a bounded wait on a bulk copy gave up
#define EPR_DEVERR_NONFINITE 4u  // NaN or Inf in the data of a solve

// Fixed-point scale of the deterministic splat: value * 2^40.
#define EPR_FX_SCALE 1099511627776.0f
#define EPR_FX_INV 9.094947017729282e-13f

// Per-plan constants handed to every kernel by value.  All per-line values
// are derived in double on the host and rounded once to float.
struct EprConsts {
    int nx, ny, ns;      // grid and number of spectral lines
    int half;            // nx / 2 (complex columns of the packed half spectrum)
    int smax;            // fast-path splat reach in pixels
    int det;             // 1 = int64 fixed-point splat accumulation
    int pdl;             // host side: launch the solver kernels with
                         // programmatic dependent launch
    int os;              // oversampling: nx, ny are the internal grid, the
                         // detector image is (ny / os) x (nx / os)
    int ovf_cap;         // overflow list entries per projection
    float inv_n;         // 1 / (nx * ny), folded into the filter
    float f[EPR_MAX_LINES];     // spectral weights, sum 1
    float mu[EPR_MAX_LINES];    // attenuation 2 k beta (1/m)
    float c[EPR_MAX_LINES];     // shift per thickness step: -L delta / p^2 (1/m)
    float wproj[EPR_MAX_LINES]; // f mu / sum(f mu^2): weights of the projection
    float ha[EPR_MAX_LINES];    // Paganin: L delta 4 pi^2 / (mu (nx p)^2)
    float hb[EPR_MAX_LINES];    // Paganin: L delta 4 pi^2 / (mu (ny p)^2)
    float qc[EPR_MAX_LINES];    // local closure: eps^2 / (4 p^4), eps = L / k
    float tneg[EPR_MAX_LINES];  // -ln 2 / mu: below it f exp(-mu T) > 2 f (splat bound)
    const float* xt;     // x-dependent spectrum: per-column constants
                         // [EPR_XT_KINDS][ns][nx] in device memory, or NULL
                         // (the uniform constants above)
};

// Kinds of the per-column table of an x-dependent spectrum.  f, mu, c, wproj
// and tneg as above, per line and detector column; the preconditioner's ha,
// hb stay per line (from the column means).
enum { EPR_XT_F = 0, EPR_XT_MU = 1, EPR_XT_C = 2, EPR_XT_WPROJ = 3, EPR_XT_TNEG = 4,
       EPR_XT_KINDS = 5 };

__device__ __forceinline__ float xt_get(const EprConsts& C, int kind, int s, int x)
{
    return __ldg(&C.xt[((size_t)kind * C.ns + s) * C.nx + x]);
}

// Per-projection solver state in device memory.
struct EprProjState {
    int done;        // 1 = converged, later iterations skip the projection
    int iters;       // iterations run
    int ovf_count[2];         // overflow list fill, by splat parity
    long long ovf_total;      // sources that took the overflow path, all iterations
    double dnorm2;            // |D|^2 of the projection (set once per solve)
    float rho, kappa;         // last values
    int pad_;
};

// Device workspace pointers (owned by the plan).
struct EprWork {
    float* P;            // [B][ny][nx]  P, or the residual D - P (mono float solve)
    float* Ps;           // [B][ns][ny][nx]        (float mode, ns > 1)
    unsigned long long* Pq;   // [B][ny][nx]       (fixed-point mode)
    unsigned long long* Psq;  // [B][ns][ny][nx]   (fixed-point mode, ns > 1)
    float2* S;           // [B][ns][ny][nx/2] packed half spectrum
    int* ovf_idx;        // [B][cap] source pixel index
    unsigned int* ovf_mask;   // [B][cap] lines that took the overflow path
    float4* ovf_tg;      // [B][cap] T and twice its gradient (x, y) at the source
    EprProjState* st;    // [B]
    double* part_a;      // [B][max_blocks] block partial sums of the inverse
    double* part_b;      // [B][max_blocks]    row pass (kappa)
    double* part_c;      // [B][max_blocks] block partial sums of the forward
                         //    row pass (rho)
    double* rho_hist;    // [B][hist_len]
    double* kappa_hist;  // [B][hist_len]
    unsigned int* err;   // device error word
    const float2* tw_x;  // twiddles exp(-2 pi i t / nx), t < nx
    const float2* tw_y;  // twiddles exp(-2 pi i t / ny), t < ny
    int hist_len;        // columns of rho_hist / kappa_hist
    int max_blocks;      // columns of part_a / part_b / part_c
    const void* col_map; // host: CUtensorMap of S for the column pass's bulk
                         // copies (NULL: the column pass uses plain loads)
    int col_radix16;     // host: 1 = the bulk-copy column pass of 2048 rows
                         // runs radix-16 stages (16, 16, 8 instead of 8, 8, 8, 4)
    int row_occ6;        // host: 1 = the one-line 2048-point row passes run six
                         // blocks per SM (40 registers) instead of five
    int col_occ5;        // host: 1 = that radix-16 column pass runs five blocks
                         // per SM (48 registers) instead of four
    int splat_occ6;      // host: 1 = the one-line residual splat runs six blocks
                         // per SM (tiles below 64 x 64, reach 3 or 4)
};

// --- small helpers ---------------------------------------------------------

// a[s] for a per-line constant array held in kernel parameters.  A runtime
// index into a by-value parameter array makes the compiler copy the array to
// local memory; selecting through compile-time indices keeps every operand a
// constant-bank read.
__device__ __forceinline__ float line_const(const float (&a)[EPR_MAX_LINES], int s)
{
    float v = a[0];
#pragma unroll
    for (int i = 1; i < EPR_MAX_LINES; ++i)
        if (s == i) v = a[i];
    return v;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// Block-wide sum of two floats; returns the totals in thread 0.
// `red` must hold 2 * 32 floats of shared memory.
__device__ __forceinline__ void block_sum2(float& a, float& b, float* red)
{
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) {
        red[wid] = a;
        red[32 + wid] = b;
    }
    __syncthreads();
    if (wid == 0) {
        a = lane < nw ? red[lane] : 0.f;
        b = lane < nw ? red[32 + lane] : 0.f;
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
        }
    }
}

// Block-wide sum of one double in a fixed order (deterministic for a fixed
// block size); the total is returned to every thread.  `red` holds 32 doubles.
__device__ __forceinline__ double block_sum_d(double v, double* red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += red[w];
    return t;
}

// Reductions over a projection without inter-block synchronisation: each
// block stores its pair of block sums in its slot of pa / pb (thread 0 holds
// them after block_sum2), with no fence and no arrival counter.  One block of
// a later kernel on the same stream, which sees every slot once its grid
// dependency wait returns, adds the slots in a fixed order (a strided walk,
// then a block tree: the same bits on every run for a given block size).
__device__ __forceinline__ void store_partials(double* pa, double* pb, float a, float b)
{
    if (threadIdx.x == 0) {
        pa[blockIdx.x] = (double)a;
        if (pb) pb[blockIdx.x] = (double)b;
    }
}

// Every thread of the block calls it; the totals reach every thread.
__device__ __forceinline__ void sum_partials(const double* pa, const double* pb, int n, double& A_out,
                                             double& B_out)
{
    __shared__ double s_red[32];
    double sa = 0.0, sb = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        sa += __ldcg(&pa[i]);
        if (pb) sb += __ldcg(&pb[i]);
    }
    A_out = block_sum_d(sa, s_red);
    B_out = pb ? block_sum_d(sb, s_red) : 0.0;
}

// kappa of iteration `it` from the n partials of the inverse row pass: the
// relative update |dT| / |T'|.  Records it, the iteration count and, at or
// below tol, the projection's convergence flag.  Every thread of the block
// calls it; the flag is visible to the whole block on return.
__device__ __forceinline__ void finalize_kappa(EprProjState* st, const double* pa, const double* pb, int n,
                                               double* hist, int hist_len, int it, float tol)
{
    double sa, sb;
    sum_partials(pa, pb, n, sa, sb);
    if (threadIdx.x == 0) {
        const double kap = sb > 0.0 ? sqrt(sa / sb) : sqrt(sa);
        st->kappa = (float)kap;
        st->iters = it + 1;
        if (hist && it < hist_len) hist[it] = kap;
        if (tol > 0.f && kap <= (double)tol) st->done = 1;
    }
    __syncthreads();
}

// rho of iteration `it` from the n partials of the forward row pass:
// |D - P| / |D|.  Every thread of the block calls it.
__device__ __forceinline__ void finalize_rho(EprProjState* st, const double* pa, int n, double* hist,
                                             int hist_len, int it)
{
    double sa, sb;
    sum_partials(pa, nullptr, n, sa, sb);
    if (threadIdx.x == 0) {
        const double dn = st->dnorm2;
        const double rho = dn > 0.0 ? sqrt(sa / dn) : sqrt(sa);
        st->rho = (float)rho;
        if (hist && it < hist_len) hist[it] = rho;
    }
}

// Programmatic dependent launch.  A kernel launched with the programmatic
// stream-serialisation attribute may start while its predecessor in the
// stream is still running.  Every kernel of the solver loop therefore
// (1) loads, before epr_grid_wait(), only data that neither its predecessor
//     nor anything later writes (D, and T in the passes after the splat),
// (2) calls epr_grid_wait(), which returns once the predecessor grid has
//     completed and its writes are visible, and only then
// (3) calls epr_grid_release(), which lets its own successor launch.
// Because of (3) at most two consecutive kernels of the loop are resident at
// once, so (1) only has to hold against the immediate predecessor.  Without
// the attribute both instructions return at once.
__device__ __forceinline__ void epr_grid_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void epr_grid_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// 16-byte asynchronous global -> shared copies (completion per thread).
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src)
{
    const unsigned int d = (unsigned int)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Kernel launch with the programmatic attribute when `pdl` is set.
template <typename... KArgs, typename... Args>
inline cudaError_t epr_launch_kernel(bool pdl, void (*kernel)(KArgs...), dim3 grid, dim3 block,
                                     size_t smem, cudaStream_t stream, Args&&... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = pdl ? at : nullptr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Launch-accounting hook (defined in epr_api.cu).
void epr_count_launch(int n);

// Let a kernel use all opt-in shared memory of the device (called once per
// device at plan creation, never while a stream is being captured).
template <typename K>
inline cudaError_t epr_allow_max_smem(K kernel)
{
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin - (int)fa.sharedSizeBytes);
}

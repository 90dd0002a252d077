// Row passes of the 2-D preconditioner FFT, fused with the steps around it.
//
// Forward row pass (R2C), one block per RP pairs of rows of one projection:
//   prologue  back-transport of the split residual (arXiv 2601.22793, Eq. 4
//             and "Iteration structure"): for every object pixel and line,
//             g_s = sum of the four bilinear weights times the residual
//             r_s = (D - P) P_s / P at the shifted corners (mono: D - P,
//             read directly when the splat stored it); or the identity
//             back-transport of the local solver; or a plain load of a real
//             map (standalone filter).  The thickness rows needed for the
//             gradient are staged in shared memory first.
//   transform two real rows packed as one complex row, z = g(y0) + i g(y1),
//             shared-memory Stockham FFT of length nx;
//   epilogue  unpack X0[k] = (Z[k] + conj Z[-k]) / 2, X1[k] = (Z[k] -
//             conj Z[-k]) / 2i and store k < nx/2 with the real Nyquist
//             value packed into the imaginary part of k = 0.
// The block also stores its share of |D - P|^2; block 0 of the column pass
// that follows adds the shares in a fixed order (deterministic) into rho.
//
// Inverse row pass (C2R), the mirror image, fused with the update
// ("Iterative inversion"): per line, I'_s = max(I_s + omega h_s, eps f_s),
// then the single-thickness projection of Eq. 7,
//   T' = - sum_s f_s mu_s ln(I'_s / f_s) / sum_s f_s mu_s^2,
// evaluated as T' = T - sum_s w_s ln(1 + omega h_s / I_s) (w_s = f_s mu_s /
// sum f mu^2), the same quantity without forming exp then log of values
// near one.  Each block stores its shares of |T' - T|^2 and |T'|^2; block 0
// of the next forward row pass (or a one-block kernel after the last
// iteration) adds them in a fixed order into kappa and retires the
// projection when kappa <= tol.
#include "epr_internal.cuh"
#include "fft.cuh"

namespace {

enum { FWD_SOLVE_NL = 0, FWD_SOLVE_LOCAL = 1, FWD_LOAD = 2 };
enum { INV_UPDATE = 0, INV_STORE = 1 };

constexpr int kEPT = 8;   // complex elements per thread in the row FFT

// Projection of a row-pass block.  The row passes walk the batch from the
// last projection to the first (grid y), the splat and the column pass from
// the first to the last: each kernel starts on the projections its
// predecessor touched last, whose data are still in L2.
__device__ __forceinline__ int row_batch_index() { return (int)(gridDim.y - 1 - blockIdx.y); }
using PR = eprfft::PadRow;  // shared layout of the packed rows
constexpr int kPad = 4;   // float2 padding between packed rows in shared memory

struct RowArgs {
    const float* T;          // [B][ny][nx]
    const float* D;          // [B][ny][nx]
    const float* P;          // [B][ny][nx]   P, or D - P when `resid`
    const float* Ps;         // [B][ns][ny][nx]
    const unsigned long long* Pq;   // fixed-point mode
    const unsigned long long* Psq;
    const float* G;          // [B][ny][nx] real input (FWD_LOAD)
    float* Out;              // [B][ny][nx] real output (INV_STORE) or T (INV_UPDATE)
    float2* S;               // [B][nl][ny][nx/2]
    EprProjState* st;
    double* part_a;          // [B][max_blocks] inverse pass partials (kappa)
    double* part_b;
    double* part_c;          // [B][max_blocks] forward pass partials (rho)
    double* hist;            // kappa history (finalised by the forward pass)
    const float2* tw;        // exp(-2 pi i t / nx)
    int RP, lgRP;            // row pairs per block
    int line0, nl;           // first physical line, number of lines handled
    int it, hist_len, max_blocks;
    int check_done;
    int fin;                 // forward: block 0 finalises kappa of iteration it - 1
    float omega, eps, tol;
};

// Block 0 of a forward solve pass (line 0) turns the inverse pass's
// partials of the previous iteration into kappa, the iteration count and
// the convergence flag, unless the projection had already converged; the
// grid dependency wait has made every partial visible.  The other blocks of
// this pass may not see the flag: a projection that converges here runs this
// pass and the splat before it once more, which changes nothing it keeps.
__device__ __forceinline__ void fwd_finalize_kappa(const RowArgs& A, int b, bool lead)
{
    if (A.fin && lead && !A.st[b].done)
        finalize_kappa(&A.st[b], A.part_a + (size_t)b * A.max_blocks,
                       A.part_b + (size_t)b * A.max_blocks, (int)gridDim.x,
                       A.hist ? A.hist + (size_t)b * A.hist_len : nullptr, A.hist_len, A.it - 1,
                       A.tol);
}

__device__ __forceinline__ int fdiv(int i, float inv_d) { return (int)(((float)i + 0.5f) * inv_d); }

template <bool DET>
__device__ __forceinline__ float ldP(const float* P, const unsigned long long* Pq, size_t i)
{
    if constexpr (DET) return (float)__ldg(&Pq[i]) * EPR_FX_INV;
    else return __ldg(&P[i]);
}

// residual of line s at detector pixel q of projection b (pb = b * npix)
template <bool DET, bool RESID>
__device__ __forceinline__ float resid(const EprConsts& C, const RowArgs& A, size_t pb, size_t q,
                                       int s)
{
    if constexpr (RESID) {   // the split residuals of the splat / split kernels
        if (C.ns == 1) return __ldg(&A.P[pb + q]);
        return __ldg(&A.Ps[pb * C.ns + (size_t)s * C.nx * C.ny + q]);
    } else {
        const float d = __ldg(&A.D[pb + q]);
        const float p = ldP<DET>(A.P, A.Pq, pb + q);
        const float r = d - p;
        if (C.ns == 1) return r;
        const size_t npix = (size_t)C.nx * C.ny;
        const size_t ps = pb * C.ns + (size_t)s * npix + q;
        const float pl = ldP<DET>(A.Ps, A.Psq, ps);
        return (p > 1e-30f) ? r * (pl / p) : r * line_const(C.f, s);
    }
}

// bilinear gather of line s's residual at (y + uy, x + ux); corners outside
// the grid read 0 (Eq. 4)
template <bool DET, bool RESID>
__device__ __forceinline__ float gather_px(const EprConsts& C, const RowArgs& A, size_t pb, int y,
                                           int x, float uy, float ux, int s)
{
    const float lim = 2.f * (float)(C.nx > C.ny ? C.nx : C.ny);
    ux = fminf(fmaxf(ux, -lim), lim);
    uy = fminf(fmaxf(uy, -lim), lim);
    const float fx = floorf(ux), fy = floorf(uy);
    const float dx = ux - fx, dy = uy - fy;
    const int cx = x + (int)fx, cy = y + (int)fy;
    const int nx = C.nx, ny = C.ny;
    const bool x0 = (unsigned)cx < (unsigned)nx, x1 = (unsigned)(cx + 1) < (unsigned)nx;
    float r00 = 0.f, r10 = 0.f, r01 = 0.f, r11 = 0.f;
    if ((unsigned)cy < (unsigned)ny) {
        const size_t row = (size_t)cy * nx;
        if (x0) r00 = resid<DET, RESID>(C, A, pb, row + cx, s);
        if (x1) r10 = resid<DET, RESID>(C, A, pb, row + cx + 1, s);
    }
    if ((unsigned)(cy + 1) < (unsigned)ny) {
        const size_t row = (size_t)(cy + 1) * nx;
        if (x0) r01 = resid<DET, RESID>(C, A, pb, row + cx, s);
        if (x1) r11 = resid<DET, RESID>(C, A, pb, row + cx + 1, s);
    }
    const float top = r00 + dx * (r10 - r00);
    const float bot = r01 + dx * (r11 - r01);
    return (1.f - dy) * top + dy * bot;
}

// XT: an x-dependent spectrum, the shift constant read per object column.
template <int MODE, bool DET, bool RESID, int NS, bool XT = false>
__global__ void __launch_bounds__(512, 2) k_row_fwd(const EprConsts C, const RowArgs A)
{
    extern __shared__ __align__(16) float2 zs[];
    __shared__ float red[64];
    const int b = row_batch_index();
    const int nx = C.nx, ny = C.ny, half = C.half;
    const int T = blockDim.x, tid = threadIdx.x;
    const int RP = A.RP, sm = nx + kPad;
    const size_t npix = (size_t)nx * ny;
    const size_t pb = (size_t)b * npix;
    const int yb = blockIdx.x * RP * 2;   // first row of the block
    const int nl = NS ? NS : A.nl;
    // thickness rows yb-1 .. yb+2RP (clamped), after the FFT buffer
    float* Ts = reinterpret_cast<float*>(zs + ((PR::len(RP * sm) + 1) & ~1));
    const int nrows = 2 * RP + 2;

    if constexpr (MODE == FWD_SOLVE_NL) {   // T is not written by the predecessor
        const float* Tb = A.T + pb;
        const int q4 = nx >> 2;
        const float inv_q4 = 1.f / (float)q4;
        for (int i = tid; i < nrows * q4; i += T) {
            const int r = fdiv(i, inv_q4), c4 = i - r * q4;
            const int gy = min(max(yb - 1 + r, 0), ny - 1);
            cp_async16(reinterpret_cast<float4*>(Ts) + i,
                       reinterpret_cast<const float4*>(Tb + (size_t)gy * nx) + c4);
        }
        cp_async_commit();
    }
    epr_grid_wait();
    if constexpr (MODE != FWD_LOAD) fwd_finalize_kappa(A, b, blockIdx.x == 0);
    if (A.check_done && A.st[b].done) {
        cp_async_wait_all();   // no copy may land after the block has left
        return;
    }
    epr_grid_release();
    if constexpr (MODE == FWD_SOLVE_NL) {
        cp_async_wait_all();
        __syncthreads();
    }

    float ra = 0.f;   // |D - P|^2 share
    const float inv_nx = 1.f / (float)nx;
    for (int sl = 0; sl < nl; ++sl) {
        const int s = A.line0 + sl;
        // prologue: packed complex input rows in shared memory
#pragma unroll 2
        for (int k = 0; k < kEPT; ++k) {
            const int e = tid + k * T;
            const int m = RP == 1 ? 0 : fdiv(e, inv_nx);
            const int x = e - m * nx;
            const int y0 = yb + 2 * m;
            float v[2];
#pragma unroll
            for (int r0 = 0; r0 < 2; ++r0) {
                const int y = y0 + r0;
                if constexpr (MODE == FWD_SOLVE_NL) {
                    const float* tr = Ts + (2 * m + r0 + 1) * nx;   // row y
                    const float t = tr[x];
                    float gx, gy;
                    if (x == 0) gx = tr[1] - t;
                    else if (x == nx - 1) gx = t - tr[x - 1];
                    else gx = 0.5f * (tr[x + 1] - tr[x - 1]);
                    if (y == 0) gy = tr[nx + x] - t;
                    else if (y == ny - 1) gy = t - tr[x - nx];
                    else gy = 0.5f * (tr[nx + x] - tr[x - nx]);
                    const float cs = XT ? xt_get(C, EPR_XT_C, s, x) : line_const(C.c, s);
                    v[r0] = gather_px<DET, RESID>(C, A, pb, y, x, cs * gy, cs * gx, s);
                } else if constexpr (MODE == FWD_SOLVE_LOCAL) {
                    v[r0] = resid<DET, RESID>(C, A, pb, (size_t)y * nx + x, s);
                } else {
                    v[r0] = __ldg(&A.G[pb + (size_t)y * nx + x]);
                }
                if constexpr (MODE != FWD_LOAD) {
                    if (sl == 0) {
                        const size_t q = (size_t)y * nx + x;
                        float r;
                        if constexpr (RESID) r = __ldg(&A.P[pb + q]);
                        else r = __ldg(&A.D[pb + q]) - ldP<DET>(A.P, A.Pq, pb + q);
                        ra += r * r;
                    }
                }
            }
            zs[PR::idx(m * sm + x)] = make_float2(v[0], v[1]);
        }
        __syncthreads();
        eprfft::fft<PR, -1, kEPT>(zs, nx, A.lgRP, 1, sm, A.tw, T, tid);
        // epilogue: unpack the two real spectra and store k < nx/2
        float2* Sb = A.S + ((size_t)b * A.nl + sl) * (size_t)ny * half;
        const float inv_half = 1.f / (float)half;
        for (int e = tid; e < RP * half; e += T) {
            const int m = RP == 1 ? 0 : fdiv(e, inv_half);
            const int k = e - m * half;
            const int y0 = yb + 2 * m;
            const int zb = m * sm;
            float2 X0, X1;
            if (k == 0) {
                const float2 z0 = zs[PR::idx(zb)], zn = zs[PR::idx(zb + half)];
                X0 = make_float2(z0.x, zn.x);
                X1 = make_float2(z0.y, zn.y);
            } else {
                const float2 a = zs[PR::idx(zb + k)], bb = cconj(zs[PR::idx(zb + nx - k)]);
                const float2 sp = cadd(a, bb), df = csub(a, bb);
                X0 = make_float2(0.5f * sp.x, 0.5f * sp.y);
                X1 = make_float2(0.5f * df.y, -0.5f * df.x);
            }
            Sb[(size_t)y0 * half + k] = X0;
            Sb[(size_t)(y0 + 1) * half + k] = X1;
        }
        __syncthreads();
    }

    if constexpr (MODE != FWD_LOAD) {   // |D - P|^2 partials; rho is formed by the column pass
        float rb = 0.f;
        block_sum2(ra, rb, red);
        store_partials(A.part_c + (size_t)b * A.max_blocks, nullptr, ra, rb);
    }
}

// ln(1 + q) for |q| < 1/4 from ln(1 + q) = 2 atanh(z), z = q / (2 + q), and
// the Taylor series of atanh: 2 z (1 + z^2/3 + z^4/5 + ... + z^10/11).  Here
// |z| < 1/7, so the first omitted term, 2 |z|^13 / 13, is below 4e-12 |z|:
// the error is the rounding of the few operations.
__device__ __forceinline__ float log1p_atanh(float q)
{
    const float z = __fdividef(q, 2.f + q);
    const float w = z * z;
    float p = fmaf(w, 1.f / 11.f, 1.f / 9.f);
    p = fmaf(w, p, 1.f / 7.f);
    p = fmaf(w, p, 1.f / 5.f);
    p = fmaf(w, p, 1.f / 3.f);
    p = fmaf(w, p, 1.f);
    return 2.f * z * p;
}

// ln(I'_s / I_s) for the update of one pixel and line, I_s = f_s exp(-mu_s t),
// I'_s = max(I_s + omega h_s, eps f_s).  With q = (omega / f_s) h_s exp(mu_s t)
// = omega h_s / I_s, the ratio is 1 + q above the floor, and
// eps f_s / I_s = eps exp(mu_s t) at it.  om_f = omega / f_s.
__device__ __forceinline__ float log_ratio(float t, float h, float om_f, float mus, float eps)
{
    const float Einv = __expf(mus * t);        // f_s / I_s
    const float q = om_f * h * Einv;
    if (1.f + q >= eps * Einv) return (fabsf(q) < 0.25f) ? log1p_atanh(q) : logf(1.f + q);
    return logf(eps) + mus * t;
}

// XT: an x-dependent spectrum, the update's constants read per column.
template <int MODE, int NS, bool XT = false>
__global__ void __launch_bounds__(512, 2) k_row_inv(const EprConsts C, const RowArgs A)
{
    extern __shared__ __align__(16) float2 zs[];
    __shared__ float red[64];
    const int b = row_batch_index();
    epr_grid_wait();
    if (A.check_done && A.st[b].done) return;
    epr_grid_release();
    const int nx = C.nx, ny = C.ny, half = C.half;
    const int T = blockDim.x, tid = threadIdx.x;
    const int RP = A.RP, sm = nx + kPad;
    const size_t npix = (size_t)nx * ny;
    const size_t pb = (size_t)b * npix;
    const int yb = blockIdx.x * RP * 2;
    const int nl = NS ? NS : A.nl;
    float* acc = reinterpret_cast<float*>(zs + ((PR::len(RP * sm) + 1) & ~1));  // [2 RP][nx]
    const float inv_nx = 1.f / (float)nx, inv_half = 1.f / (float)half;
    float da = 0.f, db = 0.f;

    for (int sl = 0; sl < nl; ++sl) {
        const int s = A.line0 + sl;
        const float2* Sb = A.S + ((size_t)b * A.nl + sl) * (size_t)ny * half;
        // unpack Z[k] = X0[k] + i X1[k] over the full row
        for (int e = tid; e < RP * half; e += T) {
            const int m = RP == 1 ? 0 : fdiv(e, inv_half);
            const int k = e - m * half;
            const int y0 = yb + 2 * m;
            const float2 s0 = Sb[(size_t)y0 * half + k];
            const float2 s1 = Sb[(size_t)(y0 + 1) * half + k];
            const int zb = m * sm;
            if (k == 0) {
                zs[PR::idx(zb)] = make_float2(s0.x, s1.x);
                zs[PR::idx(zb + half)] = make_float2(s0.y, s1.y);
            } else {
                zs[PR::idx(zb + k)] = make_float2(s0.x - s1.y, s0.y + s1.x);
                zs[PR::idx(zb + nx - k)] = make_float2(s0.x + s1.y, s1.x - s0.y);
            }
        }
        __syncthreads();
        eprfft::fft<PR, +1, kEPT>(zs, nx, A.lgRP, 1, sm, A.tw, T, tid);
#pragma unroll 2
        for (int k = 0; k < kEPT; ++k) {
            const int e = tid + k * T;
            const int m = RP == 1 ? 0 : fdiv(e, inv_nx);
            const int x = e - m * nx;
            const float2 h = zs[PR::idx(m * sm + x)];
            const size_t q0 = pb + (size_t)(yb + 2 * m) * nx + x;
            if constexpr (MODE == INV_UPDATE) {
                const float fs = XT ? xt_get(C, EPR_XT_F, s, x) : line_const(C.f, s);
                const float mus = XT ? xt_get(C, EPR_XT_MU, s, x) : line_const(C.mu, s);
                const float w = XT ? xt_get(C, EPR_XT_WPROJ, s, x) : line_const(C.wproj, s);
                const float om_f = A.omega / fs;
                const float t0 = A.Out[q0], t1 = A.Out[q0 + nx];
                const float l0 = w * log_ratio(t0, h.x, om_f, mus, A.eps);
                const float l1 = w * log_ratio(t1, h.y, om_f, mus, A.eps);
                if (nl == 1) {
                    const float n0 = t0 - l0, n1 = t1 - l1;
                    A.Out[q0] = n0;
                    A.Out[q0 + nx] = n1;
                    da += l0 * l0 + l1 * l1;
                    db += n0 * n0 + n1 * n1;
                } else {
                    float* a0 = acc + (2 * m) * nx + x;
                    if (sl == 0) {
                        a0[0] = l0;
                        a0[nx] = l1;
                    } else {
                        a0[0] += l0;
                        a0[nx] += l1;
                    }
                }
            } else {
                A.Out[q0] = h.x;
                A.Out[q0 + nx] = h.y;
            }
        }
        __syncthreads();
    }

    if constexpr (MODE == INV_UPDATE) {
        if (nl > 1) {
            for (int k = 0; k < kEPT; ++k) {
                const int e = tid + k * T;
                const int m = RP == 1 ? 0 : fdiv(e, inv_nx);
                const int x = e - m * nx;
                const size_t q0 = pb + (size_t)(yb + 2 * m) * nx + x;
                const float l0 = acc[(2 * m) * nx + x], l1 = acc[(2 * m + 1) * nx + x];
                const float n0 = A.Out[q0] - l0, n1 = A.Out[q0 + nx] - l1;
                A.Out[q0] = n0;
                A.Out[q0 + nx] = n1;
                da += l0 * l0 + l1 * l1;
                db += n0 * n0 + n1 * n1;
            }
        }
        block_sum2(da, db, red);   // kappa partials, finalised by the next forward pass
        store_partials(A.part_a + (size_t)b * A.max_blocks, A.part_b + (size_t)b * A.max_blocks, da,
                       db);
    }
}

// |D|^2 per projection, deterministic: block partials, then a fixed-order sum
__global__ void __launch_bounds__(256) k_sumsq_part(const float* __restrict__ D, size_t npix,
                                                    double* part, int max_blocks)
{
    __shared__ float red[64];
    const int b = blockIdx.y;
    const float4* Db = reinterpret_cast<const float4*>(D + (size_t)b * npix);
    const size_t n4 = npix / 4;
    float a = 0.f, z = 0.f;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4;
         i += (size_t)gridDim.x * blockDim.x) {
        const float4 v = __ldg(&Db[i]);
        a += v.x * v.x + v.y * v.y + v.z * v.z + v.w * v.w;
    }
    block_sum2(a, z, red);
    if (threadIdx.x == 0) part[(size_t)b * max_blocks + blockIdx.x] = (double)a;
}

// A NaN or an infinity anywhere in D makes the sum non-finite (finite float
// squares cannot overflow a double sum): flagged in the device error word.
__global__ void k_sumsq_final(const double* part, int nparts, int max_blocks, double scale,
                              EprProjState* st, unsigned int* err)
{
    const int b = blockIdx.x;
    if (threadIdx.x != 0) return;
    double s = 0.0;
    for (int i = 0; i < nparts; ++i) s += part[(size_t)b * max_blocks + i];
    st[b].dnorm2 = s * scale;
    if (!isfinite(s)) atomicOr(err, EPR_DEVERR_NONFINITE);
}

// ---------------------------------------------------------------------------
// Monochromatic float solve, compile-time row length NX and RP row pairs per
// block: the same passes as k_row_fwd / k_row_inv (modes FWD_SOLVE_NL with
// the residual stored by the splat, INV_UPDATE with one line) on the
// compile-time FFT engine.
// ---------------------------------------------------------------------------
template <int NX>
__host__ __device__ constexpr int ct_lg(int v) { return v <= 1 ? 0 : 1 + ct_lg<NX>(v / 2); }

// packed row pair of element e (0 <= e < NX RP); NX may be 3 * 2^k with RP = 1
template <int NX, int RP>
__device__ __forceinline__ int row_of(int e) { return RP == 1 ? 0 : (int)((unsigned)e / NX); }

// Shared memory: the thickness rows yb - 1 .. yb + 2 RP, staged for the
// gradient, alias the FFT rows, which are written only after the last
// thickness read (row_fwd_mono_smem).  256-thread monochromatic blocks run
// five per SM (48 registers).
//
// OCC6: six 256-thread blocks per SM (40 registers) instead of five: better
// in a batch of projections, worse for one (the autotuner decides).
// XT: an x-dependent spectrum, the shift constant of each object column from
// the plan's table.
template <int NX, int RP, bool POLY, bool GATHER, bool OCC6 = false, bool XT = false, int EPT = kEPT>
__global__ void __launch_bounds__(NX * RP / EPT, OCC6 ? 6 : (NX * RP / EPT == 256 && !POLY) ? 5 : (65536 / 64) / (NX * RP / EPT))
k_row_fwd_mono(const EprConsts C, const RowArgs A)
{
    constexpr int T = NX * RP / EPT;
    constexpr int MAXR = EPT >= 16 ? 16 : 8;   // radix-16 stages with 16 elements per thread
    // 16 elements per thread (8192-point rows): the thickness is read through
    // L1 instead of staged, which leaves room for two blocks per SM
    constexpr bool kStageT = EPT == kEPT;
    constexpr int SM = NX + kPad;
    constexpr int HALF = NX / 2;
    constexpr int LGRP = ct_lg<NX>(RP);
    extern __shared__ __align__(16) float2 zs[];
    __shared__ float red[64];
    const int b = row_batch_index();
    const int sl = POLY ? (int)blockIdx.z : 0;   // line of this block (polychromatic)
    const int ny = C.ny, tid = threadIdx.x;
    const size_t npix = (size_t)NX * ny;
    const size_t pb = (size_t)b * npix;
    const int yb = blockIdx.x * RP * 2;
    float* Ts = reinterpret_cast<float*>(zs);   // aliases the FFT rows (see above)
    if constexpr (GATHER && kStageT) {   // T is not written by the predecessor: fetch it before the wait
        const float* Tb = A.T + pb;
        constexpr int Q4 = NX / 4;
        constexpr int NROWS = 2 * RP + 2;
#pragma unroll
        for (int i0 = 0; i0 < NROWS * Q4; i0 += T) {
            const int i = i0 + tid;
            if (NROWS * Q4 % T == 0 || i < NROWS * Q4) {
                const int r = i / Q4, c4 = i % Q4;
                const int gy = min(max(yb - 1 + r, 0), ny - 1);
                cp_async16(reinterpret_cast<float4*>(Ts) + i,
                           reinterpret_cast<const float4*>(Tb + (size_t)gy * NX) + c4);
            }
        }
        cp_async_commit();
    }
    epr_grid_wait();
    fwd_finalize_kappa(A, b, blockIdx.x == 0 && sl == 0);
    if (A.check_done && A.st[b].done) {
        cp_async_wait_all();   // no copy may land after the block has left
        return;
    }
    cp_async_wait_all();
    __syncthreads();
    const float cs = POLY ? line_const(C.c, A.line0 + sl) : C.c[0];
    // residual D - P (one line) or the line's split residual
    const float* Rb = POLY ? A.Ps + (pb * C.ns + (size_t)(A.line0 + sl) * npix) : A.P + pb;
    const float* Rt = A.P + pb;   // D - P, for |D - P|^2
    float ra = 0.f;
    float2 vk[EPT];   // the packed row pair values, stored once the thickness is dead
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
        const int e = tid + k * T;
        const int m = row_of<NX, RP>(e), x = e - m * NX;
        const int y0 = yb + 2 * m;
        float v[2];
#pragma unroll
        for (int r0 = 0; r0 < 2; ++r0) {
            const int y = y0 + r0;
            if constexpr (!GATHER) {   // identity back-transport of the local closure
                v[r0] = __ldg(Rb + (size_t)y * NX + x);
            } else {
            const float* tr = kStageT ? Ts + (2 * m + r0 + 1) * NX : A.T + pb + (size_t)y * NX;
            const float t = kStageT ? tr[x] : __ldg(tr + x);
            // edges (one-sided differences): with one row pair per block only
            // the first and last element of a thread can be an edge column,
            // and only the first (last) row of the pair the top (bottom) row
            const bool xlo = (RP > 1 || k == 0) && x == 0;
            const bool xhi = (RP > 1 || k == EPT - 1) && x == NX - 1;
            const bool ylo = r0 == 0 && y == 0, yhi = r0 == 1 && y == ny - 1;
            float gx, gy;
            if (xlo) gx = tr[1] - t;
            else if (xhi) gx = t - tr[x - 1];
            else gx = 0.5f * (tr[x + 1] - tr[x - 1]);
            if (ylo) gy = tr[NX + x] - t;
            else if (yhi) gy = t - tr[x - NX];
            else gy = 0.5f * (tr[NX + x] - tr[x - NX]);   // rows y - 1 and y + 1 exist here
            const float lim = 2.f * (float)(NX > ny ? NX : ny);
            const float csx = XT ? xt_get(C, EPR_XT_C, A.line0 + sl, x) : cs;
            const float ux = fminf(fmaxf(csx * gx, -lim), lim);
            const float uy = fminf(fmaxf(csx * gy, -lim), lim);
            const float fx = floorf(ux), fy = floorf(uy);
            const float dx = ux - fx, dy = uy - fy;
            const int cx = x + (int)fx, cy = y + (int)fy;
            const bool x0 = (unsigned)cx < (unsigned)NX, x1 = (unsigned)(cx + 1) < (unsigned)NX;
            float r00 = 0.f, r10 = 0.f, r01 = 0.f, r11 = 0.f;
            if ((unsigned)cy < (unsigned)ny) {
                const float* rr = Rb + (size_t)cy * NX + cx;
                if (x0) r00 = __ldg(rr);
                if (x1) r10 = __ldg(rr + 1);
            }
            if ((unsigned)(cy + 1) < (unsigned)ny) {
                const float* rr = Rb + (size_t)(cy + 1) * NX + cx;
                if (x0) r01 = __ldg(rr);
                if (x1) r11 = __ldg(rr + 1);
            }
            const float top = r00 + dx * (r10 - r00);
            const float bot = r01 + dx * (r11 - r01);
            v[r0] = (1.f - dy) * top + dy * bot;
            }
            if (!POLY || sl == 0) {
                const float own = __ldg(Rt + (size_t)y * NX + x);
                ra += own * own;
            }
        }
        vk[k] = make_float2(v[0], v[1]);
    }
    if constexpr (GATHER && kStageT) __syncthreads();   // every thickness read is done
    if constexpr (RP == 1 && eprfft::ct_radix(NX, 0, MAXR) == EPT) {
        // one row pair: vk[k] = element tid + k T, the first stage's operands
        eprfft::stage0_regs<PR, -1, NX, EPT, 1, MAXR>(vk, zs, tid);
        eprfft::fft_ct<PR, -1, NX, EPT, LGRP, 1, SM, 1, MAXR>(zs, A.tw, tid);
    } else {
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
            const int e = tid + k * T;
            const int m = row_of<NX, RP>(e), x = e - m * NX;
            zs[PR::idx(m * SM + x)] = vk[k];
        }
        __syncthreads();
        eprfft::fft_ct<PR, -1, NX, EPT, LGRP, 1, SM, 0, MAXR>(zs, A.tw, tid);
    }
    epr_grid_release();
    float2* Sb = A.S + ((size_t)b * A.nl + sl) * (size_t)ny * HALF;
#pragma unroll 2
    for (int i0 = 0; i0 < RP * HALF; i0 += T) {
        const int e = i0 + tid;
        const int m = e / HALF, k = e % HALF;
        const int y0 = yb + 2 * m;
        const int zb = m * SM;
        float2 X0, X1;
        if (k == 0) {
            const float2 z0 = zs[PR::idx(zb)], zn = zs[PR::idx(zb + HALF)];
            X0 = make_float2(z0.x, zn.x);
            X1 = make_float2(z0.y, zn.y);
        } else {
            const float2 a = zs[PR::idx(zb + k)], bb = cconj(zs[PR::idx(zb + NX - k)]);
            const float2 sp = cadd(a, bb), df = csub(a, bb);
            X0 = make_float2(0.5f * sp.x, 0.5f * sp.y);
            X1 = make_float2(0.5f * df.y, -0.5f * df.x);
        }
        Sb[(size_t)y0 * HALF + k] = X0;
        Sb[(size_t)(y0 + 1) * HALF + k] = X1;
    }
    if (POLY && sl != 0) return;   // the residual norm is line 0's
    float rb = 0.f;
    block_sum2(ra, rb, red);   // |D - P|^2 partials; rho is formed by the column pass
    store_partials(A.part_c + (size_t)b * A.max_blocks, nullptr, ra, rb);
}

// The update of one result of the last inverse stage of a one-line block:
// element e = m SM + x holds rows 2m and 2m + 1 of the block at column x;
// T' = T - w ln(I'/I) from the staged thickness rows, stored, with the kappa
// partial sums kept in the functor (its call sites are inlined, so they stay
// in registers).
template <int NX, int SM, int RP, bool XT, bool STAGED = true>
struct InvUpdate1 {
    const EprConsts& C;
    const float* Tsh;      // [2 RP][NX] thickness rows of the block (STAGED), else unused
    float* out;            // T at the block's first row (read there when not STAGED)
    float mus, w, om_f, omega, eps;
    mutable float da, db;
    __device__ __forceinline__ float2 operator()(float2 h, int e) const
    {
        const int m = RP == 1 ? 0 : e / SM;
        const int x = e - m * SM;
        float* o = out + (size_t)(2 * m) * NX + x;
        const float t0 = STAGED ? Tsh[(2 * m) * NX + x] : o[0];
        const float t1 = STAGED ? Tsh[(2 * m + 1) * NX + x] : o[NX];
        float wx = w, omx = om_f, mux = mus;
        if constexpr (XT) {
            wx = xt_get(C, EPR_XT_WPROJ, 0, x);
            mux = xt_get(C, EPR_XT_MU, 0, x);
            omx = omega / xt_get(C, EPR_XT_F, 0, x);
        }
        const float l0 = wx * log_ratio(t0, h.x, omx, mux, eps);
        const float l1 = wx * log_ratio(t1, h.y, omx, mux, eps);
        const float n0 = t0 - l0, n1 = t1 - l1;
        o[0] = n0;
        o[NX] = n1;
        da += l0 * l0 + l1 * l1;
        db += n0 * n0 + n1 * n1;
        return h;
    }
};

// five 256-thread blocks per SM (48 registers): its shared memory is the FFT
// rows and 2 RP thickness rows only (row_inv_mono_smem).  EPT = 16 (8192-point
// rows): radix-16 stages, and the update reads T through L1 instead of staging
// it, so two 512-thread blocks fit on an SM.
template <int NX, int RP, bool OCC6 = false, bool XT = false, int EPT = kEPT>
__global__ void __launch_bounds__(NX * RP / EPT, OCC6 ? 6 : NX * RP / EPT == 256 ? 5 : (65536 / 64) / (NX * RP / EPT))
k_row_inv_mono(const EprConsts C, const RowArgs A)
{
    constexpr int T = NX * RP / EPT;
    constexpr int MAXR = EPT >= 16 ? 16 : 8;
    constexpr bool kStageT = EPT == kEPT;
    constexpr int SM = NX + kPad;
    constexpr int HALF = NX / 2;
    constexpr int LGRP = ct_lg<NX>(RP);
    extern __shared__ __align__(16) float2 zs[];
    __shared__ float red[64];
    const int b = row_batch_index();
    const int ny = C.ny, tid = threadIdx.x;
    const size_t pb = (size_t)b * NX * ny;
    const int yb = blockIdx.x * RP * 2;
    // rows yb .. yb + 2RP - 1 of T, copied while the spectrum is transformed
    float* Tsh = reinterpret_cast<float*>(zs + ((PR::len(RP * SM) + 1) & ~1));
    if constexpr (kStageT) {
        constexpr int Q4 = 2 * RP * NX / 4;
        const float4* src = reinterpret_cast<const float4*>(A.Out + pb + (size_t)yb * NX);
#pragma unroll
        for (int i0 = 0; i0 < Q4; i0 += T) {
            const int i = i0 + tid;
            if (Q4 % T == 0 || i < Q4) cp_async16(reinterpret_cast<float4*>(Tsh) + i, src + i);
        }
        cp_async_commit();
    }
    epr_grid_wait();
    if (A.check_done && A.st[b].done) {
        cp_async_wait_all();
        return;
    }
    const float2* Sb = A.S + (size_t)b * (size_t)ny * HALF;
#pragma unroll 2
    for (int i0 = 0; i0 < RP * HALF; i0 += T) {
        const int e = i0 + tid;
        const int m = e / HALF, k = e % HALF;
        const int y0 = yb + 2 * m;
        const float2 s0 = Sb[(size_t)y0 * HALF + k];
        const float2 s1 = Sb[(size_t)(y0 + 1) * HALF + k];
        const int zb = m * SM;
        if (k == 0) {
            zs[PR::idx(zb)] = make_float2(s0.x, s1.x);
            zs[PR::idx(zb + HALF)] = make_float2(s0.y, s1.y);
        } else {
            zs[PR::idx(zb + k)] = make_float2(s0.x - s1.y, s0.y + s1.x);
            zs[PR::idx(zb + NX - k)] = make_float2(s0.x + s1.y, s1.x - s0.y);
        }
    }
    __syncthreads();
    constexpr int NST = eprfft::ct_n_stages(NX, MAXR);
    eprfft::fft_ct_stages<PR, +1, NX, EPT, LGRP, 1, SM, 0, NST - 1, MAXR>(zs, A.tw, tid);
    epr_grid_release();
    cp_async_wait_all();   // the thickness rows: visible to all after the last stage's barrier
    // the last stage hands each result to the update (no store, no barrier)
    const InvUpdate1<NX, SM, RP, XT, kStageT> up{C, Tsh, A.Out + pb + (size_t)yb * NX, C.mu[0],
                                                 C.wproj[0], A.omega / C.f[0], A.omega, A.eps,
                                                 0.f, 0.f};
    eprfft::fft_ct_last<PR, false, false, PR, +1, NX, EPT, LGRP, 1, SM, MAXR>(zs, A.tw, tid, up);
    float da = up.da, db = up.db;
    block_sum2(da, db, red);   // kappa partials, finalised by the next forward pass
    store_partials(A.part_a + (size_t)b * A.max_blocks, A.part_b + (size_t)b * A.max_blocks, da, db);
}

// The per-line step of the polychromatic update, applied to each result of
// a line's last inverse stage (element e = m SM + x: rows 2m, 2m + 1 at
// column x): w_s ln(I'_s / I_s) added to the pixel's sum in shared memory
// (the element-to-thread map of the last stage is the same for every line,
// so each thread reads and writes its own pixels only); on the last line
// T' = T - sum is stored instead, with the kappa partial sums.
template <int NX, int SM, int RP, bool XT>
struct InvUpdatePoly {
    const EprConsts& C;
    const float* Tsh;      // [2 RP][NX] thickness rows of the block
    float* acc;            // [2 RP][NX] sums over the lines so far
    float* out;            // T at the block's first row
    int s;                 // line of this pass
    bool first, last;
    float mus, w, om_f, omega, eps;
    mutable float da, db;
    __device__ __forceinline__ float2 operator()(float2 h, int e) const
    {
        const int m = RP == 1 ? 0 : e / SM;
        const int x = e - m * SM;
        const int i0 = (2 * m) * NX + x;
        float wx = w, omx = om_f, mux = mus;
        if constexpr (XT) {
            wx = xt_get(C, EPR_XT_WPROJ, s, x);
            mux = xt_get(C, EPR_XT_MU, s, x);
            omx = omega / xt_get(C, EPR_XT_F, s, x);
        }
        const float t0 = Tsh[i0], t1 = Tsh[i0 + NX];
        float l0 = wx * log_ratio(t0, h.x, omx, mux, eps);
        float l1 = wx * log_ratio(t1, h.y, omx, mux, eps);
        if (!first) {
            l0 = acc[i0] + l0;
            l1 = acc[i0 + NX] + l1;
        }
        if (last) {
            const float n0 = t0 - l0, n1 = t1 - l1;
            float* o = out + (size_t)(2 * m) * NX + x;
            o[0] = n0;
            o[NX] = n1;
            da += l0 * l0 + l1 * l1;
            db += n0 * n0 + n1 * n1;
        } else {
            acc[i0] = l0;
            acc[i0 + NX] = l1;
        }
        return h;
    }
};

// Polychromatic update on the compile-time engine: for each line, the C2R
// rows of its filtered spectrum and w_s ln(I'_s / I_s), accumulated per
// pixel in shared memory (each thread owns its pixels); then T' = T - sum
// and the kappa partial sums.
template <int NX, int RP, bool XT = false>
__global__ void __launch_bounds__(NX * RP / kEPT, (65536 / 64) / (NX * RP / kEPT))
k_row_inv_poly(const EprConsts C, const RowArgs A)
{
    constexpr int T = NX * RP / kEPT;
    constexpr int SM = NX + kPad;
    constexpr int HALF = NX / 2;
    constexpr int LGRP = ct_lg<NX>(RP);
    extern __shared__ __align__(16) float2 zs[];
    __shared__ float red[64];
    const int b = row_batch_index();
    const int ny = C.ny, tid = threadIdx.x;
    const size_t pb = (size_t)b * NX * ny;
    const int yb = blockIdx.x * RP * 2;
    float* Tsh = reinterpret_cast<float*>(zs + ((PR::len(RP * SM) + 1) & ~1));   // [2 RP][NX]
    float* acc = Tsh + 2 * RP * NX;                                              // [2 RP][NX]
    {
        constexpr int Q4 = 2 * RP * NX / 4;
        const float4* src = reinterpret_cast<const float4*>(A.Out + pb + (size_t)yb * NX);
#pragma unroll
        for (int i0 = 0; i0 < Q4; i0 += T) {
            const int i = i0 + tid;
            if (Q4 % T == 0 || i < Q4) cp_async16(reinterpret_cast<float4*>(Tsh) + i, src + i);
        }
        cp_async_commit();
    }
    epr_grid_wait();
    if (A.check_done && A.st[b].done) {
        cp_async_wait_all();
        return;
    }
    InvUpdatePoly<NX, SM, RP, XT> up{C, Tsh, acc, A.Out + pb + (size_t)yb * NX, 0, true, false,
                                     0.f, 0.f, 0.f, A.omega, A.eps, 0.f, 0.f};
    for (int sl = 0; sl < A.nl; ++sl) {
        const int s = A.line0 + sl;
        const float2* Sb = A.S + ((size_t)b * A.nl + sl) * (size_t)ny * HALF;
#pragma unroll 2
        for (int i0 = 0; i0 < RP * HALF; i0 += T) {
            const int e = i0 + tid;
            const int m = e / HALF, k = e % HALF;
            const int y0 = yb + 2 * m;
            const float2 s0 = Sb[(size_t)y0 * HALF + k];
            const float2 s1 = Sb[(size_t)(y0 + 1) * HALF + k];
            const int zb = m * SM;
            if (k == 0) {
                zs[PR::idx(zb)] = make_float2(s0.x, s1.x);
                zs[PR::idx(zb + HALF)] = make_float2(s0.y, s1.y);
            } else {
                zs[PR::idx(zb + k)] = make_float2(s0.x - s1.y, s0.y + s1.x);
                zs[PR::idx(zb + NX - k)] = make_float2(s0.x + s1.y, s1.x - s0.y);
            }
        }
        __syncthreads();
        constexpr int NST = eprfft::ct_n_stages(NX);
        eprfft::fft_ct_stages<PR, +1, NX, kEPT, LGRP, 1, SM, 0, NST - 1>(zs, A.tw, tid);
        if (sl == 0) {
            epr_grid_release();
            cp_async_wait_all();   // the thickness rows: visible after the last stage's barrier
        }
        // the last stage adds the line's term to each thread's own pixels;
        // after its barrier nothing reads zs, so the next unpack may follow
        up.s = s;
        up.first = sl == 0;
        up.last = sl == A.nl - 1;
        up.mus = line_const(C.mu, s);
        up.w = line_const(C.wproj, s);
        up.om_f = A.omega / line_const(C.f, s);
        eprfft::fft_ct_last<PR, false, false, PR, +1, NX, kEPT, LGRP, 1, SM>(zs, A.tw, tid, up);
    }
    float da = up.da, db = up.db;
    block_sum2(da, db, red);   // kappa partials, finalised by the next forward pass
    store_partials(A.part_a + (size_t)b * A.max_blocks, A.part_b + (size_t)b * A.max_blocks, da, db);
}

// dynamic shared memory of k_row_fwd_mono: FFT rows aliased with the
// 2 RP + 2 staged thickness rows
size_t row_fwd_mono_smem(int nx, int rp)
{
    const size_t fft = (size_t)((PR::len(rp * (nx + kPad)) + 1) & ~1) * sizeof(float2);
    const size_t ts = (size_t)(2 * rp + 2) * nx * sizeof(float);
    return fft > ts ? fft : ts;
}

// dynamic shared memory of the FFT rows alone (the 16-elements-per-thread
// kernels, which stage no thickness rows)
size_t row_fft_smem(int nx, int rp)
{
    return (size_t)((PR::len(rp * (nx + kPad)) + 1) & ~1) * sizeof(float2);
}

// dynamic shared memory of k_row_inv_mono: FFT rows, T rows
size_t row_inv_mono_smem(int nx, int rp)
{
    return (size_t)((PR::len(rp * (nx + kPad)) + 1) & ~1) * sizeof(float2) +
           (size_t)(2 * rp * nx) * sizeof(float);
}

// dynamic shared memory of k_row_inv_poly: FFT rows, T rows, accumulators
size_t row_inv_poly_smem(int nx, int rp)
{
    return (size_t)((PR::len(rp * (nx + kPad)) + 1) & ~1) * sizeof(float2) +
           (size_t)2 * (2 * rp * nx) * sizeof(float);
}

// launch a specialised mono kernel when nx has one; returns false otherwise
// The compile-time row kernels with per-column constants (x-dependent
// spectrum) for the common row lengths; false when nx has none.
template <bool FWD>
bool launch_xt_ct(int nx, int rp, dim3 grid, cudaStream_t stream, const EprConsts& C,
                  const RowArgs& A, cudaError_t& err)
{
    const bool poly = A.nl > 1;
#define EPR_XT_CASE(NXV, RPV)                                                                 \
    if (nx == NXV && rp == RPV) {                                                             \
        const dim3 blk(NXV * RPV / kEPT);                                                     \
        if (FWD && !poly)                                                                     \
            err = epr_launch_kernel(C.pdl != 0, k_row_fwd_mono<NXV, RPV, false, true, false, true>, \
                                    grid, blk, row_fwd_mono_smem(NXV, RPV), stream, C, A);     \
        else if (FWD)                                                                         \
            err = epr_launch_kernel(C.pdl != 0, k_row_fwd_mono<NXV, RPV, true, true, false, true>, \
                                    dim3(grid.x, grid.y, A.nl), blk, row_fwd_mono_smem(NXV, RPV), \
                                    stream, C, A);                                            \
        else if (!poly)                                                                       \
            err = epr_launch_kernel(C.pdl != 0, k_row_inv_mono<NXV, RPV, false, true>, grid, blk, \
                                    row_inv_mono_smem(NXV, RPV), stream, C, A);               \
        else                                                                                  \
            err = epr_launch_kernel(C.pdl != 0, k_row_inv_poly<NXV, RPV, true>, grid, blk,     \
                                    row_inv_poly_smem(NXV, RPV), stream, C, A);               \
        return true;                                                                          \
    }
    EPR_XT_CASE(1024, 2)
    EPR_XT_CASE(2048, 1)
    EPR_XT_CASE(4096, 1)
#undef EPR_XT_CASE
    return false;
}

template <bool FWD, bool GATHER = true>
bool launch_mono_ct(int nx, int rp, dim3 grid, size_t smem, cudaStream_t stream, const EprConsts& C,
                    const RowArgs& A, cudaError_t& err, bool W_occ6 = false)
{
    // one line: the mono kernels; several: forward with a line per grid z,
    // inverse looping over the lines
    const bool poly = A.nl > 1;
#define EPR_MONO_CASE(NXV, RPV)                                                              \
    if (nx == NXV && rp == RPV) {                                                            \
        const dim3 blk(NXV * RPV / kEPT);                                                    \
        if (FWD && !poly) {                                                                  \
            err = epr_launch_kernel(C.pdl != 0, k_row_fwd_mono<NXV, RPV, false, GATHER>, grid, blk, \
                                    row_fwd_mono_smem(NXV, RPV), stream, C, A);              \
        } else if (FWD) {                                                                    \
            const dim3 g3(grid.x, grid.y, A.nl);                                             \
            err = epr_launch_kernel(C.pdl != 0, k_row_fwd_mono<NXV, RPV, true, GATHER>, g3, blk, \
                                    row_fwd_mono_smem(NXV, RPV), stream, C, A);              \
        } else if (!poly) {                                                                  \
            err = epr_launch_kernel(C.pdl != 0, k_row_inv_mono<NXV, RPV>, grid, blk,          \
                                    row_inv_mono_smem(NXV, RPV), stream, C, A);              \
        } else {                                                                             \
            err = epr_launch_kernel(C.pdl != 0, k_row_inv_poly<NXV, RPV>, grid, blk,          \
                                    row_inv_poly_smem(NXV, RPV), stream, C, A);              \
        }                                                                                    \
        return true;                                                                         \
    }
    EPR_MONO_CASE(256, 8)
    EPR_MONO_CASE(512, 4)
    EPR_MONO_CASE(1024, 2)
    EPR_MONO_CASE(1536, 1)
    if (nx == 2048 && rp == 1 && !poly && GATHER && W_occ6) {   // six blocks per SM
        if (FWD)
            err = epr_launch_kernel(C.pdl != 0, k_row_fwd_mono<2048, 1, false, true, true>, grid,
                                    dim3(256), row_fwd_mono_smem(2048, 1), stream, C, A);
        else
            err = epr_launch_kernel(C.pdl != 0, k_row_inv_mono<2048, 1, true>, grid, dim3(256),
                                    row_inv_mono_smem(2048, 1), stream, C, A);
        return true;
    }
    EPR_MONO_CASE(2048, 1)
    EPR_MONO_CASE(3072, 1)
    EPR_MONO_CASE(4096, 1)
    if (nx == 8192 && rp == 1 && !poly && (!FWD || GATHER)) {   // 16 per thread, two blocks per SM
        if (FWD)
            err = epr_launch_kernel(C.pdl != 0, k_row_fwd_mono<8192, 1, false, true, false, false, 16>,
                                    grid, dim3(512), row_fft_smem(8192, 1), stream, C, A);
        else
            err = epr_launch_kernel(C.pdl != 0, k_row_inv_mono<8192, 1, false, false, 16>, grid,
                                    dim3(512), row_fft_smem(8192, 1), stream, C, A);
        return true;
    }
    EPR_MONO_CASE(8192, 1)
#undef EPR_MONO_CASE
    return false;
}

template <typename K>
cudaError_t allow(K k) { return epr_allow_max_smem(k); }

cudaError_t init_mono_ct()
{
    cudaError_t e = cudaSuccess;
#define EPR_MONO_INIT(NXV, RPV)                                                  \
    if (e == cudaSuccess) e = allow(k_row_fwd_mono<NXV, RPV, false, true>);       \
    if (e == cudaSuccess) e = allow(k_row_fwd_mono<NXV, RPV, true, true>);        \
    if (e == cudaSuccess) e = allow(k_row_fwd_mono<NXV, RPV, false, false>);      \
    if (e == cudaSuccess) e = allow(k_row_fwd_mono<NXV, RPV, true, false>);       \
    if (e == cudaSuccess) e = allow(k_row_inv_mono<NXV, RPV>);                    \
    if (e == cudaSuccess) e = allow(k_row_inv_poly<NXV, RPV>);
    EPR_MONO_INIT(256, 8)
    EPR_MONO_INIT(512, 4)
    EPR_MONO_INIT(1024, 2)
    EPR_MONO_INIT(1536, 1)
    EPR_MONO_INIT(2048, 1)
    if (e == cudaSuccess) e = allow(k_row_fwd_mono<2048, 1, false, true, true>);
    if (e == cudaSuccess) e = allow(k_row_inv_mono<2048, 1, true>);
#define EPR_XT_INIT(NXV, RPV)                                                        \
    if (e == cudaSuccess) e = allow(k_row_fwd_mono<NXV, RPV, false, true, false, true>); \
    if (e == cudaSuccess) e = allow(k_row_fwd_mono<NXV, RPV, true, true, false, true>);  \
    if (e == cudaSuccess) e = allow(k_row_inv_mono<NXV, RPV, false, true>);              \
    if (e == cudaSuccess) e = allow(k_row_inv_poly<NXV, RPV, true>);
    EPR_XT_INIT(1024, 2)
    EPR_XT_INIT(2048, 1)
    EPR_XT_INIT(4096, 1)
#undef EPR_XT_INIT
    EPR_MONO_INIT(3072, 1)
    EPR_MONO_INIT(4096, 1)
    EPR_MONO_INIT(8192, 1)
    if (e == cudaSuccess) e = allow(k_row_fwd_mono<8192, 1, false, true, false, false, 16>);
    if (e == cudaSuccess) e = allow(k_row_inv_mono<8192, 1, false, false, 16>);
#undef EPR_MONO_INIT
    return e;
}

}  // namespace

struct EprRowLaunch {
    int RP, lgRP, threads;
    size_t smem;
};

EprRowLaunch epr_row_config(const EprConsts& C)
{
    EprRowLaunch L;
    int rp = 1;
    while (rp * 2 * C.nx <= 2048 && (C.ny / 2) % (rp * 2) == 0) rp *= 2;
    L.RP = rp;
    L.lgRP = 0;
    while ((1 << L.lgRP) < rp) ++L.lgRP;
    L.threads = C.nx * rp / kEPT;
    // FFT rows, then the staged thickness rows (forward) or line accumulators
    // (inverse); the larger of the two
    const size_t extra = (size_t)(2 * rp + 2) * C.nx * sizeof(float);
    L.smem = (size_t)((PR::len(rp * (C.nx + kPad)) + 1) & ~1) * sizeof(float2) + extra;  // EPR_ROW_SMEM
    return L;
}

// mode: 0 = non-local solve, 1 = local solve, 2 = load real map G.
// FWD_SOLVE_NL reads the residual D - P from P and the split residuals from P_s.
// In a solve (it > 0) block 0 also finalises kappa of iteration it - 1
// against tol.
cudaError_t epr_launch_row_fwd(const EprConsts& C, const EprWork& W, int mode, const float* T,
                               const float* D, const float* G, int line0, int nl, int it,
                               float tol, int batch, int check_done, cudaStream_t stream)
{
    const EprRowLaunch L = epr_row_config(C);
    RowArgs A = {};
    A.T = T; A.D = D; A.G = G;
    A.P = W.P; A.Ps = W.Ps; A.Pq = W.Pq; A.Psq = W.Psq;
    A.S = W.S; A.st = W.st; A.part_a = W.part_a; A.part_b = W.part_b; A.part_c = W.part_c;
    A.hist = W.kappa_hist; A.hist_len = W.hist_len; A.max_blocks = W.max_blocks;
    A.tw = W.tw_x; A.RP = L.RP; A.lgRP = L.lgRP; A.line0 = line0; A.nl = nl; A.it = it;
    A.check_done = check_done;
    A.fin = mode != FWD_LOAD && it > 0;
    A.tol = tol;
    const dim3 grid(C.ny / (2 * L.RP), batch), blk(L.threads);
    const bool mono = nl == 1, pdl = C.pdl != 0;
    cudaError_t e = cudaSuccess;
    auto go = [&](auto kernel) { e = epr_launch_kernel(pdl, kernel, grid, blk, L.smem, stream, C, A); };
    if (mode == FWD_SOLVE_NL && C.xt) {   // per-column shift constants
        if (!launch_xt_ct<true>(C.nx, L.RP, grid, stream, C, A, e))
            go(k_row_fwd<FWD_SOLVE_NL, false, true, 0, true>);
    } else if (mode == FWD_SOLVE_NL) {
        // the residual D - P is in P and, with several lines, the split
        // residuals in P_s (written by the splat flush or the split kernel)
        if (!launch_mono_ct<true>(C.nx, L.RP, grid, L.smem, stream, C, A, e, W.row_occ6 != 0)) {
            if (mono) go(k_row_fwd<FWD_SOLVE_NL, false, true, 1>);
            else go(k_row_fwd<FWD_SOLVE_NL, false, true, 0>);
        }
    } else if (mode == FWD_SOLVE_LOCAL) {
        // identity back-transport: the split residuals at the pixel itself
        if (!launch_mono_ct<true, false>(C.nx, L.RP, grid, L.smem, stream, C, A, e))
            go(k_row_fwd<FWD_SOLVE_LOCAL, false, true, 0>);
    } else {
        go(k_row_fwd<FWD_LOAD, false, false, 1>);
    }
    epr_count_launch(1);
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t epr_launch_row_inv(const EprConsts& C, const EprWork& W, int mode, float* Out,
                               int line0, int nl, int it, float omega, float eps, float tol,
                               int batch, int check_done, cudaStream_t stream)
{
    const EprRowLaunch L = epr_row_config(C);
    RowArgs A = {};
    A.Out = Out; A.S = W.S; A.st = W.st; A.part_a = W.part_a; A.part_b = W.part_b;
    A.hist_len = W.hist_len; A.max_blocks = W.max_blocks;
    A.tw = W.tw_x; A.RP = L.RP; A.lgRP = L.lgRP; A.line0 = line0; A.nl = nl; A.it = it;
    A.omega = omega; A.eps = eps; A.tol = tol; A.check_done = check_done;
    const dim3 grid(C.ny / (2 * L.RP), batch), blk(L.threads);
    const bool pdl = C.pdl != 0;
    cudaError_t e = cudaSuccess;
    auto go = [&](auto kernel) { e = epr_launch_kernel(pdl, kernel, grid, blk, L.smem, stream, C, A); };
    if (mode == INV_UPDATE && C.xt) {   // per-column update constants
        if (!launch_xt_ct<false>(C.nx, L.RP, grid, stream, C, A, e))
            go(k_row_inv<INV_UPDATE, 0, true>);
    } else if (mode == INV_UPDATE) {
        if (launch_mono_ct<false>(C.nx, L.RP, grid, L.smem, stream, C, A, e, W.row_occ6 != 0)) {
        } else if (nl == 1) go(k_row_inv<INV_UPDATE, 1>);
        else go(k_row_inv<INV_UPDATE, 0>);
    } else {
        go(k_row_inv<INV_STORE, 1>);
    }
    epr_count_launch(1);
    return e != cudaSuccess ? e : cudaGetLastError();
}

// |D|^2 of each projection into the solver state (two small launches).
// |D|^2 of each projection (D of npix pixels) times scale, into the solver
// state (two small launches).
cudaError_t epr_launch_dnorm(const EprConsts& C, const EprWork& W, const float* D, int batch,
                             size_t npix, double scale, cudaStream_t stream)
{
    const int parts = W.max_blocks < 64 ? W.max_blocks : 64;
    k_sumsq_part<<<dim3(parts, batch), 256, 0, stream>>>(D, npix, W.part_a, W.max_blocks);
    k_sumsq_final<<<batch, 32, 0, stream>>>(W.part_a, parts, W.max_blocks, scale, W.st, W.err);
    epr_count_launch(2);
    return cudaGetLastError();
}

// Blocks of a row pass (the number of partials a reduction adds up).
int epr_row_blocks(const EprConsts& C) { return C.ny / (2 * epr_row_config(C).RP); }

namespace {

// kappa of the last iteration of a solve (the forward pass of a following
// iteration finalises the others): one block per projection.
__global__ void __launch_bounds__(256) k_finalize_kappa(EprProjState* st, const double* part_a,
                                                        const double* part_b, int max_blocks,
                                                        int nblk, double* hist, int hist_len,
                                                        int it, float tol)
{
    const int b = blockIdx.x;
    epr_grid_wait();
    if (st[b].done) return;   // converged earlier: the partials are stale
    finalize_kappa(&st[b], part_a + (size_t)b * max_blocks, part_b + (size_t)b * max_blocks, nblk,
                   hist ? hist + (size_t)b * hist_len : nullptr, hist_len, it, tol);
}

}  // namespace

cudaError_t epr_launch_finalize_kappa(const EprConsts& C, const EprWork& W, int it, float tol,
                                      int batch, cudaStream_t stream)
{
    const cudaError_t e =
        epr_launch_kernel(C.pdl != 0, k_finalize_kappa, dim3(batch), dim3(256), 0, stream, W.st,
                          (const double*)W.part_a, (const double*)W.part_b, W.max_blocks,
                          epr_row_blocks(C), W.kappa_hist, W.hist_len, it, tol);
    epr_count_launch(1);
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t epr_row_init()
{
    cudaError_t e = epr_allow_max_smem(k_row_fwd<FWD_SOLVE_NL, true, false, 1>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_row_fwd<FWD_SOLVE_NL, true, false, 0>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_row_fwd<FWD_SOLVE_NL, false, true, 1>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_row_fwd<FWD_SOLVE_NL, false, false, 1>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_row_fwd<FWD_SOLVE_NL, false, false, 0>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_row_fwd<FWD_SOLVE_LOCAL, false, true, 0>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_row_fwd<FWD_LOAD, false, false, 1>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_row_inv<INV_UPDATE, 1>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_row_inv<INV_UPDATE, 0>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_row_inv<INV_STORE, 1>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_row_fwd<FWD_SOLVE_NL, false, true, 0, true>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_row_inv<INV_UPDATE, 0, true>);
    if (e == cudaSuccess) e = init_mono_ct();
    return e;
}

// Row passes of the 2-D preconditioner FFT, fused with the steps around it.
//
// Forward row pass (R2C), one block per RP pairs of rows of one projection:
//   prologue  back-transport of the split residual (arXiv 2601.22793, Eq. 4
//             and "Iteration structure"): for every object pixel and line,
//             g_s = sum of the four bilinear weights times
//             r_s(corner) = (D - P) P_s / P at the shifted corners
//             (mono: D - P); or the identity back-transport of the local
//             solver; or a plain load of a real map (standalone filter);
//   transform two real rows packed as one complex row, z = g(y0) + i g(y1),
//             shared-memory Stockham FFT of length nx;
//   epilogue  unpack X0[k] = (Z[k] + conj Z[-k]) / 2, X1[k] = (Z[k] -
//             conj Z[-k]) / 2i and store k < nx/2 with the real Nyquist
//             value packed into the imaginary part of k = 0.
// The block also adds its share of |D - P|^2 and |D|^2; the last block of a
// projection reduces the shares in a fixed order (deterministic) into rho.
//
// Inverse row pass (C2R), the mirror image, fused with the update
// ("Iterative inversion"): per line, I'_s = max(I_s + omega h_s, eps f_s),
// then the single-thickness projection of Eq. 7,
//   T' = - sum_s f_s mu_s ln(I'_s / f_s) / sum_s f_s mu_s^2,
// evaluated as T' = T - sum_s w_s ln(1 + omega h_s / I_s) (w_s = f_s mu_s /
// sum f mu^2), which is the same quantity without forming exp then log of
// values near one.  The last block of a projection reduces |T' - T|^2 and
// |T'|^2 into kappa and retires the projection when kappa <= tol.
#include "epr_internal.cuh"
#include "fft.cuh"

namespace {

enum { FWD_SOLVE_NL = 0, FWD_SOLVE_LOCAL = 1, FWD_LOAD = 2 };
enum { INV_UPDATE = 0, INV_STORE = 1 };

constexpr int kEPT = 8;   // complex elements per thread in the row FFT
constexpr int kPad = 4;   // float2 padding between packed rows in shared memory

struct RowArgs {
    const float* T;          // [B][ny][nx]
    const float* D;          // [B][ny][nx]
    const float* P;          // [B][ny][nx]          float mode
    const float* Ps;         // [B][ns][ny][nx]
    const unsigned long long* Pq;   // fixed-point mode
    const unsigned long long* Psq;
    const float* G;          // [B][ny][nx] real input (FWD_LOAD)
    float* Out;              // [B][ny][nx] real output (INV_STORE) or T (INV_UPDATE)
    float2* S;               // [B][nl][ny][nx/2]
    EprProjState* st;
    double* part_a;
    double* part_b;
    double* hist;            // rho (forward) or kappa (inverse) history
    const float2* tw;        // exp(-2 pi i t / nx)
    int RP, lgRP;            // row pairs per block
    int line0, nl;           // first physical line, number of lines handled
    int it, hist_len, max_blocks;
    int check_done;
    float omega, eps, tol;
};

template <bool DET>
__device__ __forceinline__ float ldP(const float* P, const unsigned long long* Pq, size_t i)
{
    if constexpr (DET) return (float)__ldg(&Pq[i]) * EPR_FX_INV;
    else return __ldg(&P[i]);
}

// residual of line s at detector pixel q: (D - P) P_s / P (mono: D - P)
template <bool DET>
__device__ __forceinline__ float resid(const EprConsts& C, const RowArgs& A, size_t pb, size_t q,
                                       int s)
{
    const float d = __ldg(&A.D[pb + q]);
    const float p = ldP<DET>(A.P, A.Pq, pb + q);
    const float r = d - p;
    if (C.ns == 1) return r;
    const size_t npix = (size_t)C.nx * C.ny;
    const size_t ps = pb * C.ns + (size_t)s * npix + q;  // pb = b * npix
    const float pl = ldP<DET>(A.Ps, A.Psq, ps);
    return (p > 1e-30f) ? r * (pl / p) : r * C.f[s];
}

// bilinear gather of line s's residual at (y + uy, x + ux); corners outside
// the grid read 0 (Eq. 4)
template <bool DET>
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
    float acc = 0.f;
    const bool x0 = cx >= 0 && cx < nx, x1 = cx + 1 >= 0 && cx + 1 < nx;
    if (cy >= 0 && cy < ny) {
        const size_t row = (size_t)cy * nx;
        if (x0) acc += (1.f - dx) * (1.f - dy) * resid<DET>(C, A, pb, row + cx, s);
        if (x1) acc += dx * (1.f - dy) * resid<DET>(C, A, pb, row + cx + 1, s);
    }
    if (cy + 1 >= 0 && cy + 1 < ny) {
        const size_t row = (size_t)(cy + 1) * nx;
        if (x0) acc += (1.f - dx) * dy * resid<DET>(C, A, pb, row + cx, s);
        if (x1) acc += dx * dy * resid<DET>(C, A, pb, row + cx + 1, s);
    }
    return acc;
}

__device__ __forceinline__ float grad_at(const float* Tb, int y, int x, int ny, int nx, bool along_x)
{
    const size_t o = (size_t)y * nx + x;
    if (along_x) {
        if (x == 0) return __ldg(&Tb[o + 1]) - __ldg(&Tb[o]);
        if (x == nx - 1) return __ldg(&Tb[o]) - __ldg(&Tb[o - 1]);
        return 0.5f * (__ldg(&Tb[o + 1]) - __ldg(&Tb[o - 1]));
    }
    if (y == 0) return __ldg(&Tb[o + nx]) - __ldg(&Tb[o]);
    if (y == ny - 1) return __ldg(&Tb[o]) - __ldg(&Tb[o - nx]);
    return 0.5f * (__ldg(&Tb[o + nx]) - __ldg(&Tb[o - nx]));
}

// deterministic last-block reduction of per-block (a, b) partial sums
__device__ __forceinline__ bool last_block_reduce(unsigned int* cnt, unsigned int nblk, double* pa,
                                                  double* pb, int blk, float a, float b,
                                                  double& A_out, double& B_out)
{
    __shared__ int s_last;
    if (threadIdx.x == 0) {
        pa[blk] = (double)a;
        pb[blk] = (double)b;
        __threadfence();
        const unsigned int prev = atomicAdd(cnt, 1u);
        s_last = (prev == nblk - 1u);
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    if (threadIdx.x == 0) {
        double sa = 0.0, sb = 0.0;
        for (unsigned int i = 0; i < nblk; ++i) {
            sa += ((volatile double*)pa)[i];
            sb += ((volatile double*)pb)[i];
        }
        A_out = sa;
        B_out = sb;
        *cnt = 0u;
    }
    return true;
}

template <int MODE, bool DET>
__global__ void __launch_bounds__(512) k_row_fwd(const EprConsts C, const RowArgs A)
{
    extern __shared__ __align__(16) float2 zs[];
    __shared__ float red[64];
    const int b = blockIdx.y;
    if (A.check_done && A.st[b].done) return;
    const int nx = C.nx, ny = C.ny, half = C.half;
    const int T = blockDim.x, tid = threadIdx.x;
    const int RP = A.RP, sm = nx + kPad;
    const size_t npix = (size_t)nx * ny;
    const size_t pb = (size_t)b * npix;
    const int yb = blockIdx.x * RP * 2;   // first row of the block
    const float* Tb = A.T ? A.T + pb : nullptr;

    // per-thread pixels: element e = tid + k T of the RP x nx packed rows
    int px[kEPT], pm[kEPT];
    float gxa[kEPT], gya[kEPT], gxb[kEPT], gyb[kEPT];
    float ra = 0.f, rb = 0.f;   // |D - P|^2, |D|^2 shares
#pragma unroll
    for (int k = 0; k < kEPT; ++k) {
        const int e = tid + k * T;
        pm[k] = e / nx;
        px[k] = e - pm[k] * nx;
        if constexpr (MODE == FWD_SOLVE_NL) {
            const int y0 = yb + 2 * pm[k];
            gxa[k] = grad_at(Tb, y0, px[k], ny, nx, true);
            gya[k] = grad_at(Tb, y0, px[k], ny, nx, false);
            gxb[k] = grad_at(Tb, y0 + 1, px[k], ny, nx, true);
            gyb[k] = grad_at(Tb, y0 + 1, px[k], ny, nx, false);
        }
        if constexpr (MODE != FWD_LOAD) {
            const int y0 = yb + 2 * pm[k];
            const size_t q0 = (size_t)y0 * nx + px[k], q1 = q0 + nx;
            const float d0 = __ldg(&A.D[pb + q0]), d1 = __ldg(&A.D[pb + q1]);
            const float r0 = d0 - ldP<DET>(A.P, A.Pq, pb + q0);
            const float r1 = d1 - ldP<DET>(A.P, A.Pq, pb + q1);
            ra += r0 * r0 + r1 * r1;
            rb += d0 * d0 + d1 * d1;
        }
    }

    for (int sl = 0; sl < A.nl; ++sl) {
        const int s = A.line0 + sl;
        // prologue: packed complex input rows in shared memory
#pragma unroll
        for (int k = 0; k < kEPT; ++k) {
            const int y0 = yb + 2 * pm[k], x = px[k];
            float v0, v1;
            if constexpr (MODE == FWD_SOLVE_NL) {
                const float cs = C.c[s];
                v0 = gather_px<DET>(C, A, pb, y0, x, cs * gya[k], cs * gxa[k], s);
                v1 = gather_px<DET>(C, A, pb, y0 + 1, x, cs * gyb[k], cs * gxb[k], s);
            } else if constexpr (MODE == FWD_SOLVE_LOCAL) {
                v0 = resid<DET>(C, A, pb, (size_t)y0 * nx + x, s);
                v1 = resid<DET>(C, A, pb, (size_t)(y0 + 1) * nx + x, s);
            } else {
                const float* Gb = A.G + pb;
                v0 = __ldg(&Gb[(size_t)y0 * nx + x]);
                v1 = __ldg(&Gb[(size_t)(y0 + 1) * nx + x]);
            }
            zs[pm[k] * sm + x] = make_float2(v0, v1);
        }
        __syncthreads();
        eprfft::fft<-1, kEPT>(zs, nx, A.lgRP, 1, sm, A.tw, T, tid);
        // epilogue: unpack the two real spectra and store k < nx/2
        float2* Sb = A.S + ((size_t)b * A.nl + sl) * (size_t)ny * half;
        for (int e = tid; e < RP * half; e += T) {
            const int m = e / half, k = e - m * half;
            const int y0 = yb + 2 * m;
            const float2* z = zs + m * sm;
            float2 X0, X1;
            if (k == 0) {
                const float2 z0 = z[0], zn = z[half];
                X0 = make_float2(z0.x, zn.x);
                X1 = make_float2(z0.y, zn.y);
            } else {
                const float2 a = z[k], bb = cconj(z[nx - k]);
                const float2 sp = cadd(a, bb), df = csub(a, bb);
                X0 = make_float2(0.5f * sp.x, 0.5f * sp.y);
                X1 = make_float2(0.5f * df.y, -0.5f * df.x);
            }
            Sb[(size_t)y0 * half + k] = X0;
            Sb[(size_t)(y0 + 1) * half + k] = X1;
        }
        __syncthreads();
    }

    if constexpr (MODE != FWD_LOAD) {
        block_sum2(ra, rb, red);
        double sa, sb;
        if (last_block_reduce(&A.st[b].cnt_fwd, gridDim.x, A.part_a + (size_t)b * A.max_blocks,
                              A.part_b + (size_t)b * A.max_blocks, blockIdx.x, ra, rb, sa, sb)) {
            if (threadIdx.x == 0) {
                const double rho = sb > 0.0 ? sqrt(sa / sb) : sqrt(sa);
                A.st[b].rho = (float)rho;
                if (A.hist && A.it < A.hist_len) A.hist[(size_t)b * A.hist_len + A.it] = rho;
            }
        }
    }
}

template <int MODE>
__global__ void __launch_bounds__(512) k_row_inv(const EprConsts C, const RowArgs A)
{
    extern __shared__ __align__(16) float2 zs[];
    __shared__ float red[64];
    const int b = blockIdx.y;
    if (A.check_done && A.st[b].done) return;
    const int nx = C.nx, ny = C.ny, half = C.half;
    const int T = blockDim.x, tid = threadIdx.x;
    const int RP = A.RP, sm = nx + kPad;
    const size_t npix = (size_t)nx * ny;
    const size_t pb = (size_t)b * npix;
    const int yb = blockIdx.x * RP * 2;

    int px[kEPT], pm[kEPT];
    float t0[kEPT], t1[kEPT], a0[kEPT], a1[kEPT];
#pragma unroll
    for (int k = 0; k < kEPT; ++k) {
        const int e = tid + k * T;
        pm[k] = e / nx;
        px[k] = e - pm[k] * nx;
        a0[k] = 0.f;
        a1[k] = 0.f;
        if constexpr (MODE == INV_UPDATE) {
            const size_t q0 = (size_t)(yb + 2 * pm[k]) * nx + px[k];
            t0[k] = A.Out[pb + q0];
            t1[k] = A.Out[pb + q0 + nx];
        }
    }

    for (int sl = 0; sl < A.nl; ++sl) {
        const int s = A.line0 + sl;
        const float2* Sb = A.S + ((size_t)b * A.nl + sl) * (size_t)ny * half;
        // unpack Z[k] = X0[k] + i X1[k] over the full row
        for (int e = tid; e < RP * half; e += T) {
            const int m = e / half, k = e - m * half;
            const int y0 = yb + 2 * m;
            const float2 s0 = Sb[(size_t)y0 * half + k];
            const float2 s1 = Sb[(size_t)(y0 + 1) * half + k];
            float2* z = zs + m * sm;
            if (k == 0) {
                z[0] = make_float2(s0.x, s1.x);
                z[half] = make_float2(s0.y, s1.y);
            } else {
                z[k] = make_float2(s0.x - s1.y, s0.y + s1.x);
                z[nx - k] = make_float2(s0.x + s1.y, s1.x - s0.y);
            }
        }
        __syncthreads();
        eprfft::fft<+1, kEPT>(zs, nx, A.lgRP, 1, sm, A.tw, T, tid);
#pragma unroll
        for (int k = 0; k < kEPT; ++k) {
            const float2 h = zs[pm[k] * sm + px[k]];
            if constexpr (MODE == INV_UPDATE) {
                // ln of the updated line intensity relative to f_s exp(-mu_s T)
                const float fs = C.f[s], mus = C.mu[s];
                float lr[2];
                const float hv[2] = {h.x, h.y}, tv[2] = {t0[k], t1[k]};
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const float E = __expf(-mus * tv[r]);          // I_s / f_s
                    const float add = A.omega * hv[r] / fs;         // omega h_s / f_s
                    const float v = E + add;                        // I'_s / f_s before the floor
                    if (v >= A.eps) {
                        const float q = add / E;
                        lr[r] = (fabsf(q) < 0.5f) ? log1pf(q) : (logf(v) + mus * tv[r]);
                    } else {
                        lr[r] = logf(A.eps) + mus * tv[r];
                    }
                }
                a0[k] += C.wproj[s] * lr[0];
                a1[k] += C.wproj[s] * lr[1];
            } else {
                a0[k] = h.x;
                a1[k] = h.y;
            }
        }
        __syncthreads();
    }

    float da = 0.f, db = 0.f;
#pragma unroll
    for (int k = 0; k < kEPT; ++k) {
        const size_t q0 = (size_t)(yb + 2 * pm[k]) * nx + px[k];
        if constexpr (MODE == INV_UPDATE) {
            const float n0 = t0[k] - a0[k], n1 = t1[k] - a1[k];
            A.Out[pb + q0] = n0;
            A.Out[pb + q0 + nx] = n1;
            da += a0[k] * a0[k] + a1[k] * a1[k];
            db += n0 * n0 + n1 * n1;
        } else {
            A.Out[pb + q0] = a0[k];
            A.Out[pb + q0 + nx] = a1[k];
        }
    }
    if constexpr (MODE == INV_UPDATE) {
        block_sum2(da, db, red);
        double sa, sb;
        if (last_block_reduce(&A.st[b].cnt_inv, gridDim.x, A.part_a + (size_t)b * A.max_blocks,
                              A.part_b + (size_t)b * A.max_blocks, blockIdx.x, da, db, sa, sb)) {
            if (threadIdx.x == 0) {
                const double kap = sb > 0.0 ? sqrt(sa / sb) : sqrt(sa);
                A.st[b].kappa = (float)kap;
                A.st[b].iters = A.it + 1;
                if (A.hist && A.it < A.hist_len) A.hist[(size_t)b * A.hist_len + A.it] = kap;
                if (A.tol > 0.f && kap <= (double)A.tol) A.st[b].done = 1;
            }
        }
    }
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
    L.smem = (size_t)rp * (C.nx + kPad) * sizeof(float2);
    return L;
}

// mode: 0 = non-local solve, 1 = local solve, 2 = load real map G
cudaError_t epr_launch_row_fwd(const EprConsts& C, const EprWork& W, int mode, const float* T,
                               const float* D, const float* G, int line0, int nl, int it,
                               int batch, int check_done, cudaStream_t stream)
{
    const EprRowLaunch L = epr_row_config(C);
    RowArgs A = {};
    A.T = T; A.D = D; A.G = G;
    A.P = W.P; A.Ps = W.Ps; A.Pq = W.Pq; A.Psq = W.Psq;
    A.S = W.S; A.st = W.st; A.part_a = W.part_a; A.part_b = W.part_b;
    A.hist = W.rho_hist; A.hist_len = W.hist_len; A.max_blocks = W.max_blocks;
    A.tw = W.tw_x; A.RP = L.RP; A.lgRP = L.lgRP; A.line0 = line0; A.nl = nl; A.it = it;
    A.check_done = check_done;
    dim3 grid(C.ny / (2 * L.RP), batch);
    // the local closure writes float maps in both accumulation modes
    if (mode == FWD_SOLVE_NL) {
        if (C.det) k_row_fwd<FWD_SOLVE_NL, true><<<grid, L.threads, L.smem, stream>>>(C, A);
        else k_row_fwd<FWD_SOLVE_NL, false><<<grid, L.threads, L.smem, stream>>>(C, A);
    } else if (mode == FWD_SOLVE_LOCAL) {
        k_row_fwd<FWD_SOLVE_LOCAL, false><<<grid, L.threads, L.smem, stream>>>(C, A);
    } else {
        k_row_fwd<FWD_LOAD, false><<<grid, L.threads, L.smem, stream>>>(C, A);
    }
    epr_count_launch(1);
    return cudaGetLastError();
}

// mode: 0 = update T in place (Out = T), 1 = store the filtered real map to Out
cudaError_t epr_launch_row_inv(const EprConsts& C, const EprWork& W, int mode, float* Out,
                               int line0, int nl, int it, float omega, float eps, float tol,
                               int batch, int check_done, cudaStream_t stream)
{
    const EprRowLaunch L = epr_row_config(C);
    RowArgs A = {};
    A.Out = Out; A.S = W.S; A.st = W.st; A.part_a = W.part_a; A.part_b = W.part_b;
    A.hist = W.kappa_hist; A.hist_len = W.hist_len; A.max_blocks = W.max_blocks;
    A.tw = W.tw_x; A.RP = L.RP; A.lgRP = L.lgRP; A.line0 = line0; A.nl = nl; A.it = it;
    A.omega = omega; A.eps = eps; A.tol = tol; A.check_done = check_done;
    dim3 grid(C.ny / (2 * L.RP), batch);
    if (mode == INV_UPDATE) k_row_inv<INV_UPDATE><<<grid, L.threads, L.smem, stream>>>(C, A);
    else k_row_inv<INV_STORE><<<grid, L.threads, L.smem, stream>>>(C, A);
    epr_count_launch(1);
    return cudaGetLastError();
}

cudaError_t epr_row_init()
{
    cudaError_t e = epr_allow_max_smem(k_row_fwd<FWD_SOLVE_NL, true>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_row_fwd<FWD_SOLVE_NL, false>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_row_fwd<FWD_SOLVE_LOCAL, false>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_row_fwd<FWD_LOAD, false>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_row_inv<INV_UPDATE>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_row_inv<INV_STORE>);
    return e;
}

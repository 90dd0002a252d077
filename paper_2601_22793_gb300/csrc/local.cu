// Local O(L^2) forward closure (arXiv 2601.22793, Eq. 1) in pixel units,
// and its diffraction-pressure term alone for the non-local model to second
// order (k_wkb1, at the end),
// per spectral line, summed over lines (Eq. 5):
//   P_s = I - D_x(I u_x) - D_y(I u_y)                                    m = 1
//       + 1/2 [D_xx(I u_x^2) + 2 D_x D_y(I u_x u_y) + D_yy(I u_y^2)]
//       - eps^2/(4 p^4) [D_x(I D_x Q) + D_y(I D_y Q)]                      m = 2
// with I = f_s exp(-mu_s T), u = c_s G[T] and Q = (D_xx + D_yy) sqrt(I) /
// sqrt(I).  D_i: central differences, one-sided at the grid edges; D_ii:
// [1, -2, 1] with the edge value replicated.  (eps grad phi = p u and the
// physical derivative is D / p, which gives these pixel-unit forms.)
//
// One block computes a 32 x 32 output tile.  The nested derivatives reach 3
// pixels, so the thickness is staged with a 3-pixel halo and every
// intermediate field is evaluated in shared memory on a halo that shrinks by
// one pixel per derivative.  Derivative stencils test the GLOBAL coordinate
// for the edge rules, so values staged outside the grid are never used by
// an in-grid output.
#include "epr_internal.cuh"

namespace {

constexpr int kLT = 32;            // output tile
constexpr int kLH = 3;             // halo
constexpr int kLE = kLT + 2 * kLH; // staged extent (38)
constexpr int kLN = kLE * kLE;
constexpr int kLocalThreads = 256;

struct LocalArgs {
    const float* T;
    float* P;       // [B][ny][nx]
    float* Ps;      // [B][ns][ny][nx] or NULL
    const EprProjState* st;
    int order;
    int check_done;
};

// Derivative stencils of a field given as a function of the staged index
// (a shared array, or a product of shared arrays formed on the fly).
template <class F>
__device__ __forceinline__ float dX(F f, int l, int gx, int nx)
{
    if (gx == 0) return f(l + 1) - f(l);
    if (gx == nx - 1) return f(l) - f(l - 1);
    return 0.5f * (f(l + 1) - f(l - 1));
}
template <class F>
__device__ __forceinline__ float dY(F f, int l, int gy, int ny)
{
    if (gy == 0) return f(l + kLE) - f(l);
    if (gy == ny - 1) return f(l) - f(l - kLE);
    return 0.5f * (f(l + kLE) - f(l - kLE));
}
template <class F>
__device__ __forceinline__ float dXX(F f, int l, int gx, int nx)
{
    const float lo = gx == 0 ? f(l) : f(l - 1);
    const float hi = gx == nx - 1 ? f(l) : f(l + 1);
    return lo - 2.f * f(l) + hi;
}
template <class F>
__device__ __forceinline__ float dYY(F f, int l, int gy, int ny)
{
    const float lo = gy == 0 ? f(l) : f(l - kLE);
    const float hi = gy == ny - 1 ? f(l) : f(l + kLE);
    return lo - 2.f * f(l) + hi;
}

struct Arr {
    const float* a;
    __device__ __forceinline__ float operator()(int l) const { return a[l]; }
};

// Shared fields: T, G_x, G_y, I (order 1); also Q, D_y(I u_x u_y), I D_x Q,
// I D_y Q (order 2).  The fluxes I u and I u u are formed inside the stencils
// from I and G.
constexpr int local_fields(int order) { return order >= 2 ? 8 : 4; }

template <int ORDER>
__global__ void __launch_bounds__(kLocalThreads) k_local(const EprConsts C, const LocalArgs A)
{
    extern __shared__ __align__(16) float sm[];
    float* Ts = sm;
    float* GX = Ts + kLN;
    float* GY = GX + kLN;
    float* I = GY + kLN;
    float* Q = I + kLN;       // order 2 only, as the three below
    float* DYB = Q + kLN;
    float* CXQ = DYB + kLN;
    float* CYQ = CXQ + kLN;

    const int nx = C.nx, ny = C.ny, ns = C.ns, b = blockIdx.z;
    epr_grid_wait();
    if (A.check_done && A.st[b].done) return;
    epr_grid_release();
    const int ty0 = blockIdx.y * kLT, tx0 = blockIdx.x * kLT;
    const int gy0 = ty0 - kLH, gx0 = tx0 - kLH;
    const size_t npix = (size_t)nx * ny;
    const float* Tb = A.T + (size_t)b * npix;
    const int tid = threadIdx.x;

    for (int i = tid; i < kLN; i += kLocalThreads) {
        const int ly = i / kLE, lx = i - ly * kLE;
        const int gy = min(max(gy0 + ly, 0), ny - 1), gx = min(max(gx0 + lx, 0), nx - 1);
        Ts[i] = __ldg(&Tb[(size_t)gy * nx + gx]);
    }
    __syncthreads();
    // gradient on the 2-pixel halo
    for (int i = tid; i < kLN; i += kLocalThreads) {
        const int ly = i / kLE, lx = i - ly * kLE;
        if (ly < 1 || ly >= kLE - 1 || lx < 1 || lx >= kLE - 1) continue;
        GX[i] = dX(Arr{Ts}, i, gx0 + lx, nx);
        GY[i] = dY(Arr{Ts}, i, gy0 + ly, ny);
    }
    __syncthreads();

    float pacc[kLT * kLT / kLocalThreads];
#pragma unroll
    for (int k = 0; k < kLT * kLT / kLocalThreads; ++k) pacc[k] = 0.f;

    for (int s = 0; s < ns; ++s) {
        const float fs = line_const(C.f, s), mus = line_const(C.mu, s);
        const float cs = line_const(C.c, s), qc = line_const(C.qc, s);
        // fluxes I u_x, I u_y and I u_i u_j at staged index j
        auto AX = [&](int j) { return I[j] * (cs * GX[j]); };
        auto AY = [&](int j) { return I[j] * (cs * GY[j]); };
        auto BXX = [&](int j) { const float ux = cs * GX[j]; return I[j] * ux * ux; };
        auto BYY = [&](int j) { const float uy = cs * GY[j]; return I[j] * uy * uy; };
        auto BXY = [&](int j) { return I[j] * (cs * GX[j]) * (cs * GY[j]); };
        for (int i = tid; i < kLN; i += kLocalThreads) I[i] = fs * __expf(-mus * Ts[i]);
        __syncthreads();
        if constexpr (ORDER >= 2) {
            // Q = (D_xx + D_yy) sqrt(I) / sqrt(I).  With sqrt(I) = sqrt(f) e^(-mu T / 2)
            // each neighbour n contributes sqrt(I_n) / sqrt(I) - 1 = expm1(-mu (T_n - T) / 2)
            // (a replicated edge neighbour contributes 0): the same quotient
            // without the cancellation of second differences of a near-constant.
            const float hm = -0.5f * mus;
            for (int i = tid; i < kLN; i += kLocalThreads) {   // 1-pixel halo
                const int ly = i / kLE, lx = i - ly * kLE;
                if (ly < 1 || ly >= kLE - 1 || lx < 1 || lx >= kLE - 1) continue;
                const int gx = gx0 + lx, gy = gy0 + ly;
                const float t = Ts[i];
                float q = 0.f;
                if (gx > 0) q += expm1f(hm * (Ts[i - 1] - t));
                if (gx < nx - 1) q += expm1f(hm * (Ts[i + 1] - t));
                if (gy > 0) q += expm1f(hm * (Ts[i - kLE] - t));
                if (gy < ny - 1) q += expm1f(hm * (Ts[i + kLE] - t));
                Q[i] = I[i] > 0.f ? q : 0.f;
            }
            __syncthreads();
            for (int i = tid; i < kLN; i += kLocalThreads) {   // 2-pixel halo
                const int ly = i / kLE, lx = i - ly * kLE;
                if (ly < 2 || ly >= kLE - 2 || lx < 2 || lx >= kLE - 2) continue;
                const int gx = gx0 + lx, gy = gy0 + ly;
                DYB[i] = dY(BXY, i, gy, ny);
                CXQ[i] = I[i] * dX(Arr{Q}, i, gx, nx);
                CYQ[i] = I[i] * dY(Arr{Q}, i, gy, ny);
            }
            __syncthreads();
        }
#pragma unroll
        for (int k = 0; k < kLT * kLT / kLocalThreads; ++k) {
            const int o = tid + k * kLocalThreads;
            const int oy = o / kLT, ox = o - oy * kLT;
            const int gy = ty0 + oy, gx = tx0 + ox;
            if (gy >= ny || gx >= nx) continue;
            const int i = (oy + kLH) * kLE + (ox + kLH);
            float p = I[i] - dX(AX, i, gx, nx) - dY(AY, i, gy, ny);
            if constexpr (ORDER >= 2) {
                p += 0.5f * (dXX(BXX, i, gx, nx) + dYY(BYY, i, gy, ny)) + dX(Arr{DYB}, i, gx, nx);
                p -= qc * (dX(Arr{CXQ}, i, gx, nx) + dY(Arr{CYQ}, i, gy, ny));
            }
            pacc[k] += p;
            if (A.Ps) A.Ps[((size_t)b * ns + s) * npix + (size_t)gy * nx + gx] = p;
        }
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < kLT * kLT / kLocalThreads; ++k) {
        const int o = tid + k * kLocalThreads;
        const int oy = o / kLT, ox = o - oy * kLT;
        const int gy = ty0 + oy, gx = tx0 + ox;
        if (gy >= ny || gx >= nx) continue;
        A.P[(size_t)b * npix + (size_t)gy * nx + gx] = pacc[k];
    }
}

// The non-local model to second order: the transport's prediction (P, P_s of
// the splat, float or fixed point) minus the diffraction-pressure term of
// Eq. 1 of every line, eps^2/(4 p^4) [D_x(I D_x Q) + D_y(I D_y Q)], with the
// line's object intensity I = f_s exp(-mu_s T) at the same pixel and the
// stencils and Q of the order-2 closure above.  Writes float P (and P_s for
// several lines); the residual split reads them.  No atomics: the result is
// the same on every run.
struct Wkb1Args {
    const float* T;
    float* P;                        // [B][ny][nx] in (float mode) and out
    float* Ps;                       // [B][ns][ny][nx] in/out (ns > 1)
    const unsigned long long* Pq;    // fixed-point sums of the splat (DET)
    const unsigned long long* Psq;
    const EprProjState* st;
    int check_done;
};

constexpr int kWkb1Fields = 5;   // T, I, Q, I D_x Q, I D_y Q

template <bool DET>
__global__ void __launch_bounds__(kLocalThreads) k_wkb1(const EprConsts C, const Wkb1Args A)
{
    extern __shared__ __align__(16) float sm[];
    float* Ts = sm;
    float* I = Ts + kLN;
    float* Q = I + kLN;
    float* CXQ = Q + kLN;
    float* CYQ = CXQ + kLN;
    const int nx = C.nx, ny = C.ny, ns = C.ns, b = blockIdx.z;
    epr_grid_wait();
    if (A.check_done && A.st[b].done) return;
    epr_grid_release();
    const int ty0 = blockIdx.y * kLT, tx0 = blockIdx.x * kLT;
    const int gy0 = ty0 - kLH, gx0 = tx0 - kLH;
    const size_t npix = (size_t)nx * ny;
    const float* Tb = A.T + (size_t)b * npix;
    const int tid = threadIdx.x;
    constexpr int KO = kLT * kLT / kLocalThreads;

    for (int i = tid; i < kLN; i += kLocalThreads) {
        const int ly = i / kLE, lx = i - ly * kLE;
        const int gy = min(max(gy0 + ly, 0), ny - 1), gx = min(max(gx0 + lx, 0), nx - 1);
        Ts[i] = __ldg(&Tb[(size_t)gy * nx + gx]);
    }
    float pacc[KO];
#pragma unroll
    for (int k = 0; k < KO; ++k) pacc[k] = 0.f;

    for (int s = 0; s < ns; ++s) {
        const float fs = line_const(C.f, s), mus = line_const(C.mu, s), qc = line_const(C.qc, s);
        __syncthreads();   // Ts staged; the previous line's fields are consumed
        for (int i = tid; i < kLN; i += kLocalThreads) I[i] = fs * __expf(-mus * Ts[i]);
        // Q on the 1-pixel halo, as the order-2 closure forms it
        const float hm = -0.5f * mus;
        for (int i = tid; i < kLN; i += kLocalThreads) {
            const int ly = i / kLE, lx = i - ly * kLE;
            if (ly < 1 || ly >= kLE - 1 || lx < 1 || lx >= kLE - 1) continue;
            const int gx = gx0 + lx, gy = gy0 + ly;
            const float t = Ts[i];
            float q = 0.f;
            if (gx > 0) q += expm1f(hm * (Ts[i - 1] - t));
            if (gx < nx - 1) q += expm1f(hm * (Ts[i + 1] - t));
            if (gy > 0) q += expm1f(hm * (Ts[i - kLE] - t));
            if (gy < ny - 1) q += expm1f(hm * (Ts[i + kLE] - t));
            Q[i] = I[i] > 0.f ? q : 0.f;   // I[i] was written by this thread
        }
        __syncthreads();
        for (int i = tid; i < kLN; i += kLocalThreads) {   // 2-pixel halo
            const int ly = i / kLE, lx = i - ly * kLE;
            if (ly < 2 || ly >= kLE - 2 || lx < 2 || lx >= kLE - 2) continue;
            const int gx = gx0 + lx, gy = gy0 + ly;
            CXQ[i] = I[i] * dX(Arr{Q}, i, gx, nx);
            CYQ[i] = I[i] * dY(Arr{Q}, i, gy, ny);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < KO; ++k) {
            const int o = tid + k * kLocalThreads;
            const int oy = o / kLT, ox = o - oy * kLT;
            const int gy = ty0 + oy, gx = tx0 + ox;
            if (gy >= ny || gx >= nx) continue;
            const int i = (oy + kLH) * kLE + (ox + kLH);
            const float term = -qc * (dX(Arr{CXQ}, i, gx, nx) + dY(Arr{CYQ}, i, gy, ny));
            pacc[k] += term;
            if (ns > 1) {
                const size_t o2 = ((size_t)b * ns + s) * npix + (size_t)gy * nx + gx;
                const float ps = DET ? (float)A.Psq[o2] * EPR_FX_INV : A.Ps[o2];
                A.Ps[o2] = ps + term;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < KO; ++k) {
        const int o = tid + k * kLocalThreads;
        const int oy = o / kLT, ox = o - oy * kLT;
        const int gy = ty0 + oy, gx = tx0 + ox;
        if (gy >= ny || gx >= nx) continue;
        const size_t o2 = (size_t)b * npix + (size_t)gy * nx + gx;
        const float p = DET ? (float)A.Pq[o2] * EPR_FX_INV : A.P[o2];
        A.P[o2] = p + pacc[k];
    }
}

}  // namespace

size_t epr_local_smem(int order) { return (size_t)local_fields(order) * kLN * sizeof(float); }

// Second-order term of the non-local model, after the splat (one launch).
// fixed_point = 1 reads the splat's integer sums.
cudaError_t epr_launch_wkb1(const EprConsts& C, const EprWork& W, const float* T, int fixed_point,
                            int batch, int check_done, cudaStream_t stream)
{
    Wkb1Args A;
    A.T = T;
    A.P = W.P;
    A.Ps = W.Ps;
    A.Pq = W.Pq;
    A.Psq = W.Psq;
    A.st = W.st;
    A.check_done = check_done;
    dim3 grid((C.nx + kLT - 1) / kLT, (C.ny + kLT - 1) / kLT, batch);
    const size_t smem = (size_t)kWkb1Fields * kLN * sizeof(float);
    const cudaError_t e =
        fixed_point ? epr_launch_kernel(C.pdl != 0, k_wkb1<true>, grid, dim3(kLocalThreads), smem,
                                        stream, C, A)
                    : epr_launch_kernel(C.pdl != 0, k_wkb1<false>, grid, dim3(kLocalThreads), smem,
                                        stream, C, A);
    epr_count_launch(1);
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t epr_launch_local(const EprConsts& C, const EprWork& W, const float* T, float* P,
                             float* Ps, int order, int batch, int check_done, cudaStream_t stream)
{
    LocalArgs A;
    A.T = T;
    A.P = P;
    A.Ps = Ps;
    A.st = W.st;
    A.order = order;
    A.check_done = check_done;
    dim3 grid((C.nx + kLT - 1) / kLT, (C.ny + kLT - 1) / kLT, batch);
    const cudaError_t e =
        order >= 2 ? epr_launch_kernel(C.pdl != 0, k_local<2>, grid, dim3(kLocalThreads),
                                       epr_local_smem(2), stream, C, A)
                   : epr_launch_kernel(C.pdl != 0, k_local<1>, grid, dim3(kLocalThreads),
                                       epr_local_smem(1), stream, C, A);
    epr_count_launch(1);
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t epr_local_init()
{
    cudaError_t e = epr_allow_max_smem(k_local<1>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_local<2>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_wkb1<false>);
    return e != cudaSuccess ? e : epr_allow_max_smem(k_wkb1<true>);
}

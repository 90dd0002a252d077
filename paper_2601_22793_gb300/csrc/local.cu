// Local O(L^2) forward closure (arXiv 2601.22793, Eq. 1) in pixel units,
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

__device__ __forceinline__ float dX(const float* F, int l, int gx, int nx)
{
    if (gx == 0) return F[l + 1] - F[l];
    if (gx == nx - 1) return F[l] - F[l - 1];
    return 0.5f * (F[l + 1] - F[l - 1]);
}
__device__ __forceinline__ float dY(const float* F, int l, int gy, int ny)
{
    if (gy == 0) return F[l + kLE] - F[l];
    if (gy == ny - 1) return F[l] - F[l - kLE];
    return 0.5f * (F[l + kLE] - F[l - kLE]);
}
__device__ __forceinline__ float dXX(const float* F, int l, int gx, int nx)
{
    const float lo = gx == 0 ? F[l] : F[l - 1];
    const float hi = gx == nx - 1 ? F[l] : F[l + 1];
    return lo - 2.f * F[l] + hi;
}
__device__ __forceinline__ float dYY(const float* F, int l, int gy, int ny)
{
    const float lo = gy == 0 ? F[l] : F[l - kLE];
    const float hi = gy == ny - 1 ? F[l] : F[l + kLE];
    return lo - 2.f * F[l] + hi;
}

__global__ void __launch_bounds__(kLocalThreads) k_local(const EprConsts C, const LocalArgs A)
{
    extern __shared__ __align__(16) float sm[];
    float* Ts = sm;
    float* GX = Ts + kLN;
    float* GY = GX + kLN;
    float* I = GY + kLN;
    float* SQ = I + kLN;
    float* AX = SQ + kLN;
    float* AY = AX + kLN;
    float* BXY = AY + kLN;
    float* BXX = BXY + kLN;
    float* BYY = BXX + kLN;
    float* Q = BYY + kLN;
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
        GX[i] = dX(Ts, i, gx0 + lx, nx);
        GY[i] = dY(Ts, i, gy0 + ly, ny);
    }
    __syncthreads();

    float pacc[kLT * kLT / kLocalThreads];
#pragma unroll
    for (int k = 0; k < kLT * kLT / kLocalThreads; ++k) pacc[k] = 0.f;

    for (int s = 0; s < ns; ++s) {
        const float fs = C.f[s], mus = C.mu[s], cs = C.c[s], qc = C.qc[s];
        for (int i = tid; i < kLN; i += kLocalThreads) {
            const float v = fs * __expf(-mus * Ts[i]);
            I[i] = v;
            SQ[i] = sqrtf(v);
        }
        __syncthreads();
        for (int i = tid; i < kLN; i += kLocalThreads) {
            const int ly = i / kLE, lx = i - ly * kLE;
            if (ly < 1 || ly >= kLE - 1 || lx < 1 || lx >= kLE - 1) continue;
            const float ux = cs * GX[i], uy = cs * GY[i], Iv = I[i];
            AX[i] = Iv * ux;
            AY[i] = Iv * uy;
            if (A.order >= 2) {
                BXY[i] = Iv * ux * uy;
                BXX[i] = Iv * ux * ux;
                BYY[i] = Iv * uy * uy;
                const float sq = SQ[i];
                const float lap = dXX(SQ, i, gx0 + lx, nx) + dYY(SQ, i, gy0 + ly, ny);
                Q[i] = sq > 0.f ? lap / sq : 0.f;
            }
        }
        __syncthreads();
        if (A.order >= 2) {
            for (int i = tid; i < kLN; i += kLocalThreads) {
                const int ly = i / kLE, lx = i - ly * kLE;
                if (ly < 2 || ly >= kLE - 2 || lx < 2 || lx >= kLE - 2) continue;
                const int gx = gx0 + lx, gy = gy0 + ly;
                DYB[i] = dY(BXY, i, gy, ny);
                CXQ[i] = I[i] * dX(Q, i, gx, nx);
                CYQ[i] = I[i] * dY(Q, i, gy, ny);
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
            if (A.order >= 2) {
                p += 0.5f * (dXX(BXX, i, gx, nx) + dYY(BYY, i, gy, ny)) + dX(DYB, i, gx, nx);
                p -= qc * (dX(CXQ, i, gx, nx) + dY(CYQ, i, gy, ny));
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

}  // namespace

size_t epr_local_smem() { return (size_t)14 * kLN * sizeof(float); }

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
    const cudaError_t e = epr_launch_kernel(C.pdl != 0, k_local, grid, dim3(kLocalThreads),
                                            epr_local_smem(), stream, C, A);
    epr_count_launch(1);
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t epr_local_init() { return epr_allow_max_smem(k_local); }

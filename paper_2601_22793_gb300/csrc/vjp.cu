// Vector-Jacobian product of the non-local forward model (not in the paper:
// the analytic transpose of the transport of Eq. 3 with the shift of Eq. 2
// and the single-thickness intensity of Eq. 7), for calibration by gradient
// descent.  With gbar = dF/dP, per line s and source pixel with mapped point
// (x + u_x, y + u_y), corner values g00, g10, g01, g11 of gbar (0 outside
// the grid) and a = M_s^* gbar there:
//   Tbar     += -mu_s I_s a                                (through I_s)
//   vx, vy   += c_s ubar_x, c_s ubar_y with
//               ubar_x = I_s [(1-d_y)(g10 - g00) + d_y (g11 - g01)],
//               ubar_y = I_s [(1-d_x)(g01 - g00) + d_x (g11 - g10)]
//               (derivative of the bilinear weights; right derivative where a
//               mapped point crosses a pixel boundary)
//   cbar_s   += ubar . G[T],   mubar_s += -T I_s a         (scalars)
// then Tbar += G^T[vx, vy], the transpose of the numpy-gradient stencil.
// The host turns cbar, mubar into dF/dL, dF/ddelta_s, dF/dbeta_s.
#include "epr_internal.cuh"

namespace {

struct VjpArgs {
    const float* T;
    const float* gbar;
    float* Tbar;         // receives -sum mu I a, then the full gradient
    float* vx;           // [B][ny][nx]
    float* vy;
    double* part;        // [B][nblk][2 ns]  (cbar_s, mubar_s) per block
    int nblk;
};

__device__ __forceinline__ float grad_v(const float* Tb, int y, int x, int ny, int nx, bool along_x)
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

constexpr int kVjpThreads = 256;

__global__ void __launch_bounds__(kVjpThreads) k_vjp_pix(const EprConsts C, const VjpArgs A)
{
    __shared__ float s_c[EPR_MAX_LINES], s_f[EPR_MAX_LINES], s_mu[EPR_MAX_LINES];
    __shared__ float red[2 * EPR_MAX_LINES][kVjpThreads / 32];
    if (threadIdx.x == 0) {
#pragma unroll
        for (int s = 0; s < EPR_MAX_LINES; ++s) {
            s_c[s] = C.c[s];
            s_f[s] = C.f[s];
            s_mu[s] = C.mu[s];
        }
    }
    __syncthreads();
    const int nx = C.nx, ny = C.ny, ns = C.ns, b = blockIdx.y;
    const size_t npix = (size_t)nx * ny, pb = (size_t)b * npix;
    const float* Tb = A.T + pb;
    const float* Gb = A.gbar + pb;
    float cacc[EPR_MAX_LINES], macc[EPR_MAX_LINES];
    for (int s = 0; s < ns; ++s) {
        cacc[s] = 0.f;
        macc[s] = 0.f;
    }
    for (size_t i = blockIdx.x * (size_t)kVjpThreads + threadIdx.x; i < npix;
         i += (size_t)gridDim.x * kVjpThreads) {
        const int y = (int)(i / nx), x = (int)(i - (size_t)y * nx);
        const float t = __ldg(&Tb[i]);
        const float gxv = grad_v(Tb, y, x, ny, nx, true), gyv = grad_v(Tb, y, x, ny, nx, false);
        const float lim = 2.f * (float)(nx > ny ? nx : ny);
        float tb = 0.f, vxs = 0.f, vys = 0.f;
        for (int s = 0; s < ns; ++s) {
            const float cs = s_c[s];
            const float ux = fminf(fmaxf(cs * gxv, -lim), lim), uy = fminf(fmaxf(cs * gyv, -lim), lim);
            const float fx = floorf(ux), fy = floorf(uy);
            const float dx = ux - fx, dy = uy - fy;
            const int cx = x + (int)fx, cy = y + (int)fy;
            const bool x0 = (unsigned)cx < (unsigned)nx, x1 = (unsigned)(cx + 1) < (unsigned)nx;
            float g00 = 0.f, g10 = 0.f, g01 = 0.f, g11 = 0.f;
            if ((unsigned)cy < (unsigned)ny) {
                const float* r = Gb + (size_t)cy * nx + cx;
                if (x0) g00 = __ldg(r);
                if (x1) g10 = __ldg(r + 1);
            }
            if ((unsigned)(cy + 1) < (unsigned)ny) {
                const float* r = Gb + (size_t)(cy + 1) * nx + cx;
                if (x0) g01 = __ldg(r);
                if (x1) g11 = __ldg(r + 1);
            }
            const float a = (1.f - dy) * ((1.f - dx) * g00 + dx * g10) + dy * ((1.f - dx) * g01 + dx * g11);
            const float Is = s_f[s] * __expf(-s_mu[s] * t);
            const float ubx = Is * ((1.f - dy) * (g10 - g00) + dy * (g11 - g01));
            const float uby = Is * ((1.f - dx) * (g01 - g00) + dx * (g11 - g10));
            tb += -s_mu[s] * Is * a;
            vxs += cs * ubx;
            vys += cs * uby;
            cacc[s] += ubx * gxv + uby * gyv;
            macc[s] += -t * Is * a;
        }
        A.Tbar[pb + i] = tb;
        A.vx[pb + i] = vxs;
        A.vy[pb + i] = vys;
    }
    // deterministic block partials: warp shuffles, then warps in order
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int s = 0; s < ns; ++s) {
        float c = cacc[s], m = macc[s];
        for (int o = 16; o > 0; o >>= 1) {
            c += __shfl_down_sync(0xffffffffu, c, o);
            m += __shfl_down_sync(0xffffffffu, m, o);
        }
        if (lane == 0) {
            red[2 * s][wid] = c;
            red[2 * s + 1][wid] = m;
        }
    }
    __syncthreads();
    if (threadIdx.x < 2 * ns) {
        double acc = 0.0;
        for (int w = 0; w < kVjpThreads / 32; ++w) acc += (double)red[threadIdx.x][w];
        A.part[((size_t)b * A.nblk + blockIdx.x) * 2 * ns + threadIdx.x] = acc;
    }
}

// transpose of the unit-spacing numpy-gradient stencil along one axis
__device__ __forceinline__ float gT1(const float* v, size_t st, int n, int x)
{
    float acc = 0.f;
    if (x - 1 >= 1 && x - 1 <= n - 2) acc += 0.5f * v[(size_t)(x - 1) * st];
    if (x + 1 >= 1 && x + 1 <= n - 2) acc -= 0.5f * v[(size_t)(x + 1) * st];
    if (x == 1) acc += v[0];
    if (x == 0) acc -= v[0];
    if (x == n - 1) acc += v[(size_t)(n - 1) * st];
    if (x == n - 2) acc -= v[(size_t)(n - 1) * st];
    return acc;
}

__global__ void k_vjp_gT(const EprConsts C, const VjpArgs A)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int b = blockIdx.z;
    const int nx = C.nx, ny = C.ny;
    if (x >= nx || y >= ny) return;
    const size_t pb = (size_t)b * nx * ny;
    const float* vx = A.vx + pb + (size_t)y * nx;
    const float* vy = A.vy + pb + x;
    const size_t o = pb + (size_t)y * nx + x;
    A.Tbar[o] += gT1(vx, 1, nx, x) + gT1(vy, (size_t)nx, ny, y);
}

}  // namespace

// Two kernels; the per-block scalar partials land in `part` ([batch][nblk][2 ns]).
cudaError_t epr_launch_vjp(const EprConsts& C, const float* T, const float* gbar, float* Tbar,
                           float* vx, float* vy, double* part, int nblk, int batch,
                           cudaStream_t stream)
{
    VjpArgs A;
    A.T = T;
    A.gbar = gbar;
    A.Tbar = Tbar;
    A.vx = vx;
    A.vy = vy;
    A.part = part;
    A.nblk = nblk;
    k_vjp_pix<<<dim3(nblk, batch), kVjpThreads, 0, stream>>>(C, A);
    k_vjp_gT<<<dim3((C.nx + 63) / 64, (C.ny + 3) / 4, batch), dim3(64, 4), 0, stream>>>(C, A);
    epr_count_launch(2);
    return cudaGetLastError();
}

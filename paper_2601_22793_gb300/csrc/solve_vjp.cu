// Reverse mode through the unrolled non-local solve (not in the paper: the
// calibration of L, delta_s and beta_s by gradient descent through a fixed
// number of iterations of "Iteration structure", with the readings R1-R7 of
// the forward solve).  Given dF/dtau_N, each iteration is recomputed from its
// stored iterate and undone step by step:
//   tau' = -num / den,  num = sum_s f_s mu_s ln(I'_s / f_s),  den = sum_s f_s mu_s^2
//   I'_s = max(I_s + omega h_s, eps_I f_s)        (no gradient through the floor)
//   h_s = F^-1 H_s F g_s                          (self-adjoint; H_s depends on
//                                                  mu_s and L delta_s)
//   g_s = M_s^* r_s                               (input adjoint: the splat of
//                                                  the field; shift: the
//                                                  derivative of the bilinear
//                                                  interpolation of r_s)
//   r_s = r P_s / P (P > 1e-30, else r f_s),  r = D - P,  P = sum_s P_s
//   P_s = M_s[I_s],  I_s = f_s exp(-mu_s tau),  u_s = c_s G[tau]
// The kernels here are the pixelwise and transport steps; the host sequence
// (epr_solve_vjp in epr_api.cu) runs them with the solver's own splat, the
// standalone gather and the preconditioner passes (the column pass also
// applies dH/dmu and dH/d(L delta)).  Per-line maps of this path are laid out
// [n_lines][B][ny][nx] so that one line of a batch is contiguous.  Scalar
// reductions store fixed-order block partials in double; k_sv_accum adds them
// into per-projection accumulators, so the scalars are the same on every run
// up to the order of the float atomics of k_sv_splat_field.
#include "epr_internal.cuh"

namespace {

constexpr int kSvThreads = 256;

// numpy.gradient along one axis at (y, x), unit spacing
__device__ __forceinline__ float sv_grad(const float* Tb, int y, int x, int ny, int nx, bool along_x)
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

// Mapped point of pixel (y, x) for shift (ux, uy): the corner 00 and the
// fractions, the shift clamped as the solver's gather clamps it.
struct Mapped {
    int cx, cy;
    float dx, dy;
};

__device__ __forceinline__ Mapped sv_map(int y, int x, float ux, float uy, int ny, int nx)
{
    const float lim = 2.f * (float)(nx > ny ? nx : ny);
    ux = fminf(fmaxf(ux, -lim), lim);
    uy = fminf(fmaxf(uy, -lim), lim);
    const float fx = floorf(ux), fy = floorf(uy);
    Mapped m;
    m.dx = ux - fx;
    m.dy = uy - fy;
    m.cx = x + (int)fx;
    m.cy = y + (int)fy;
    return m;
}

// the four corner values of e at a mapped point (0 outside the grid)
__device__ __forceinline__ void sv_corners(const float* e, const Mapped& m, int ny, int nx, float& g00,
                                           float& g10, float& g01, float& g11)
{
    const bool x0 = (unsigned)m.cx < (unsigned)nx, x1 = (unsigned)(m.cx + 1) < (unsigned)nx;
    g00 = g10 = g01 = g11 = 0.f;
    if ((unsigned)m.cy < (unsigned)ny) {
        const float* r = e + (size_t)m.cy * nx + m.cx;
        if (x0) g00 = __ldg(r);
        if (x1) g10 = __ldg(r + 1);
    }
    if ((unsigned)(m.cy + 1) < (unsigned)ny) {
        const float* r = e + (size_t)(m.cy + 1) * nx + m.cx;
        if (x0) g01 = __ldg(r);
        if (x1) g11 = __ldg(r + 1);
    }
}

// Block sum of up to NV floats per thread into double partials
// part[(b * nblk + block) * nslot + slot0 + k], in a fixed order.
template <int NV>
__device__ __forceinline__ void sv_block_partials(float (&v)[NV], int nv, double* part, int nblk,
                                                  int nslot, int slot0, int b)
{
    __shared__ float red[NV][kSvThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        if (k >= nv) break;
        float a = v[k];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) red[k][wid] = a;
    }
    __syncthreads();
    if (threadIdx.x < nv) {
        double acc = 0.0;
        for (int w = 0; w < kSvThreads / 32; ++w) acc += (double)red[threadIdx.x][w];
        part[((size_t)b * nblk + blockIdx.x) * nslot + slot0 + threadIdx.x] = acc;
    }
}

// r = D - P and r_s = r P_s / P (P > 1e-30), else r f_s; P_s of one line is P.
__global__ void __launch_bounds__(kSvThreads) k_sv_split(const EprConsts C, const float* D, const float* P,
                                                         const float* Ps, float* r, float* RS, int B)
{
    const int b = blockIdx.y, ns = C.ns;
    const size_t npix = (size_t)C.nx * C.ny, pb = (size_t)b * npix;
    for (size_t q = blockIdx.x * (size_t)kSvThreads + threadIdx.x; q < npix;
         q += (size_t)gridDim.x * kSvThreads) {
        const float p = P[pb + q];
        const float rr = __ldg(&D[pb + q]) - p;
        r[pb + q] = rr;
        for (int s = 0; s < ns; ++s) {
            const float ps = ns > 1 ? Ps[(pb * ns) + (size_t)s * npix + q] : p;
            RS[((size_t)s * B + b) * npix + q] = p > 1e-30f ? rr * (ps / p) : rr * line_const(C.f, s);
        }
    }
}

// The projection, floor and log of the update, backwards.  From tbar = dF/dtau'
// per pixel: numbar = -tbar / den; HB_s = omega Ibar'_s with Ibar'_s = numbar
// f_s mu_s / I'_s above the floor, 0 at it.  Partials (slots): 0 = sum tbar num
// / den^2 (the denominator's share, turned into mu_s terms on the host),
// 1 + s = sum numbar f_s ln(I'_s / f_s).
__global__ void __launch_bounds__(kSvThreads) k_sv_update_adj(const EprConsts C, const float* T,
                                                              const float* Hs, const float* tb,
                                                              float* HB, double* part, int nblk,
                                                              int B, float omega, float eps,
                                                              float inv_den)
{
    const int b = blockIdx.y, ns = C.ns;
    const size_t npix = (size_t)C.nx * C.ny, pb = (size_t)b * npix;
    float acc[EPR_MAX_LINES + 1];
#pragma unroll
    for (int k = 0; k < EPR_MAX_LINES + 1; ++k) acc[k] = 0.f;
    for (size_t q = blockIdx.x * (size_t)kSvThreads + threadIdx.x; q < npix;
         q += (size_t)gridDim.x * kSvThreads) {
        const float t = __ldg(&T[pb + q]);
        const float tbar = __ldg(&tb[pb + q]);
        float num = 0.f;
        for (int s = 0; s < ns; ++s) {
            const float fs = line_const(C.f, s), mus = line_const(C.mu, s);
            const float Is = fs * __expf(-mus * t);
            const float In = Is + omega * __ldg(&Hs[((size_t)s * B + b) * npix + q]);
            const float Ic = fmaxf(In, eps * fs);
            num += fs * mus * logf(Ic / fs);
        }
        const float numb = -tbar * inv_den;
        acc[0] += tbar * num * inv_den * inv_den;
        for (int s = 0; s < ns; ++s) {
            const float fs = line_const(C.f, s), mus = line_const(C.mu, s);
            const float Is = fs * __expf(-mus * t);
            const float In = Is + omega * __ldg(&Hs[((size_t)s * B + b) * npix + q]);
            const float fl = eps * fs;
            const float Ic = fmaxf(In, fl);
            acc[1 + s] += numb * fs * logf(Ic / fs);
            const float Inb = In < fl ? 0.f : numb * fs * mus / Ic;
            HB[((size_t)s * B + b) * npix + q] = omega * Inb;
        }
    }
    sv_block_partials<EPR_MAX_LINES + 1>(acc, ns + 1, part, nblk, ns + 1, 0, b);
}

// sum a b per projection (partials in slot 0)
__global__ void __launch_bounds__(kSvThreads) k_sv_dot(const float* a, const float* bm, size_t npix,
                                                       double* part, int nblk)
{
    const int b = blockIdx.y;
    const size_t pb = (size_t)b * npix;
    float acc[1] = {0.f};
    for (size_t q = blockIdx.x * (size_t)kSvThreads + threadIdx.x; q < npix;
         q += (size_t)gridDim.x * kSvThreads)
        acc[0] += __ldg(&a[pb + q]) * __ldg(&bm[pb + q]);
    sv_block_partials<1>(acc, 1, part, nblk, 1, 0, b);
}

// out += M_s[field]: the bilinear redistribution of a signed field at the
// shift of line s (the adjoint of the gather), with float atomics.
__global__ void __launch_bounds__(kSvThreads) k_sv_splat_field(const EprConsts C, const float* T,
                                                               const float* field, float* out, int s)
{
    const int b = blockIdx.y, nx = C.nx, ny = C.ny;
    const size_t npix = (size_t)nx * ny, pb = (size_t)b * npix;
    const float* Tb = T + pb;
    const float cs = line_const(C.c, s);
    for (size_t q = blockIdx.x * (size_t)kSvThreads + threadIdx.x; q < npix;
         q += (size_t)gridDim.x * kSvThreads) {
        const float v = __ldg(&field[pb + q]);
        if (v == 0.f) continue;
        const int y = (int)(q / nx), x = (int)(q - (size_t)y * nx);
        const Mapped m = sv_map(y, x, cs * sv_grad(Tb, y, x, ny, nx, true),
                                cs * sv_grad(Tb, y, x, ny, nx, false), ny, nx);
        const bool x0 = (unsigned)m.cx < (unsigned)nx, x1 = (unsigned)(m.cx + 1) < (unsigned)nx;
        float* o = out + pb;
        if ((unsigned)m.cy < (unsigned)ny) {
            const size_t row = (size_t)m.cy * nx;
            if (x0) atomicAdd(o + row + m.cx, v * (1.f - m.dx) * (1.f - m.dy));
            if (x1) atomicAdd(o + row + m.cx + 1, v * m.dx * (1.f - m.dy));
        }
        if ((unsigned)(m.cy + 1) < (unsigned)ny) {
            const size_t row = (size_t)(m.cy + 1) * nx;
            if (x0) atomicAdd(o + row + m.cx, v * (1.f - m.dx) * m.dy);
            if (x1) atomicAdd(o + row + m.cx + 1, v * m.dx * m.dy);
        }
    }
}

// Shift derivatives of the bilinear interpolation of e (line s) at every
// object pixel: dux = (1-dy)(g10-g00) + dy(g11-g01), duy = (1-dx)(g01-g00) +
// dx(g11-g10) (the right derivative at a pixel boundary), times a multiplier
// w; vx += c_s w dux, vy += c_s w duy and partial slot 0 += w (dux G_x + duy
// G_y) (dF/dc_s).
//   MODE 0 (the gather's shift): e = r_s, w = gbar_s.
//   MODE 1 (the splat's shift and input): e = Pbar_s, w = I_s; also Ibar_s =
//     HB_s / omega + interp(e) gives tn += -mu_s I_s Ibar_s and partial slot 1
//     += -T I_s Ibar_s (dF/dmu_s).
template <int MODE>
__global__ void __launch_bounds__(kSvThreads) k_sv_interp_du(const EprConsts C, const float* T,
                                                             const float* e, const float* wmap,
                                                             const float* HB, float* vx, float* vy,
                                                             float* tn, double* part, int nblk,
                                                             int s, float inv_omega)
{
    const int b = blockIdx.y, nx = C.nx, ny = C.ny;
    const size_t npix = (size_t)nx * ny, pb = (size_t)b * npix;
    const float* Tb = T + pb;
    const float cs = line_const(C.c, s), fs = line_const(C.f, s), mus = line_const(C.mu, s);
    float acc[2] = {0.f, 0.f};
    for (size_t q = blockIdx.x * (size_t)kSvThreads + threadIdx.x; q < npix;
         q += (size_t)gridDim.x * kSvThreads) {
        const int y = (int)(q / nx), x = (int)(q - (size_t)y * nx);
        const float gx = sv_grad(Tb, y, x, ny, nx, true), gy = sv_grad(Tb, y, x, ny, nx, false);
        const Mapped m = sv_map(y, x, cs * gx, cs * gy, ny, nx);
        float g00, g10, g01, g11;
        sv_corners(e + pb, m, ny, nx, g00, g10, g01, g11);
        const float dux = (1.f - m.dy) * (g10 - g00) + m.dy * (g11 - g01);
        const float duy = (1.f - m.dx) * (g01 - g00) + m.dx * (g11 - g10);
        float w;
        if constexpr (MODE == 0) {
            w = __ldg(&wmap[pb + q]);
        } else {
            const float t = __ldg(&Tb[q]);
            w = fs * __expf(-mus * t);   // I_s
            const float val = (1.f - m.dy) * ((1.f - m.dx) * g00 + m.dx * g10) +
                              m.dy * ((1.f - m.dx) * g01 + m.dx * g11);
            const float Ib = __ldg(&HB[pb + q]) * inv_omega + val;
            tn[pb + q] += -mus * w * Ib;
            acc[1] += -t * w * Ib;
        }
        vx[pb + q] += cs * w * dux;
        vy[pb + q] += cs * w * duy;
        acc[0] += w * (dux * gx + duy * gy);
    }
    sv_block_partials<2>(acc, MODE == 0 ? 1 : 2, part, nblk, 2, 0, b);
}

// The residual split backwards, per pixel (every line at once): from rbar_s
// (in RSB, overwritten by Pbar_s), with P, P_s and r of the iteration:
//   rbar = sum_s rbar_s P_s / P (P > 1e-30; else sum_s rbar_s f_s),
//   Pbar = -sum_s rbar_s r P_s / P^2 - rbar,  Pbar_s = rbar_s r / P + Pbar,
// and Dbar += rbar.
__global__ void __launch_bounds__(kSvThreads) k_sv_split_adj(const EprConsts C, float* RSB,
                                                             const float* P, const float* Ps,
                                                             const float* r, float* Db, int B)
{
    const int b = blockIdx.y, ns = C.ns;
    const size_t npix = (size_t)C.nx * C.ny, pb = (size_t)b * npix;
    for (size_t q = blockIdx.x * (size_t)kSvThreads + threadIdx.x; q < npix;
         q += (size_t)gridDim.x * kSvThreads) {
        const float p = P[pb + q], rr = r[pb + q];
        const bool pos = p > 1e-30f;
        float rbar = 0.f, pbar = 0.f;
        for (int s = 0; s < ns; ++s) {
            const float rsb = RSB[((size_t)s * B + b) * npix + q];
            const float ps = ns > 1 ? Ps[(pb * ns) + (size_t)s * npix + q] : p;
            if (pos) {
                rbar += rsb * (ps / p);
                pbar -= rsb * rr * ps / (p * p);
            } else {
                rbar += rsb * line_const(C.f, s);
            }
        }
        Db[pb + q] += rbar;
        pbar -= rbar;
        for (int s = 0; s < ns; ++s) {
            const size_t o = ((size_t)s * B + b) * npix + q;
            const float rsb = RSB[o];
            RSB[o] = (pos ? rsb * rr / p : 0.f) + pbar;
        }
    }
}

// transpose of the unit-spacing numpy-gradient stencil along one axis
__device__ __forceinline__ float sv_gT1(const float* v, size_t st, int n, int x)
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

// tn += G^T [vx, vy]
__global__ void k_sv_gT(const EprConsts C, const float* vx, const float* vy, float* tn)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int b = blockIdx.z, nx = C.nx, ny = C.ny;
    if (x >= nx || y >= ny) return;
    const size_t pb = (size_t)b * nx * ny;
    tn[pb + (size_t)y * nx + x] += sv_gT1(vx + pb + (size_t)y * nx, 1, nx, x) +
                                   sv_gT1(vy + pb + x, (size_t)nx, ny, y);
}

// acc[b * nacc + slot_acc] += scale * sum_{blk < nused} part[(b * nblk + blk) *
// nslot + slot], one block per projection, in a fixed order
__global__ void __launch_bounds__(256) k_sv_accum(const double* part, int nblk, int nused, int nslot,
                                                  int slot, double* acc, int nacc, int slot_acc,
                                                  double scale)
{
    __shared__ double red[32];
    const int b = blockIdx.x;
    double v = 0.0;
    for (int k = threadIdx.x; k < nused; k += blockDim.x)
        v += part[((size_t)b * nblk + k) * nslot + slot];
    const double t = block_sum_d(v, red);
    if (threadIdx.x == 0) acc[(size_t)b * nacc + slot_acc] += scale * t;
}

inline dim3 sv_grid(size_t npix, int nblk, int batch)
{
    size_t blocks = (npix + kSvThreads - 1) / kSvThreads;
    if (blocks > (size_t)nblk) blocks = nblk;
    return dim3((unsigned)blocks, batch);
}

}  // namespace

// Blocks per projection of the reductions (the partial buffers hold this many).
int epr_sv_blocks() { return 608; }   // 4 per SM on 152 SMs

cudaError_t epr_launch_sv_split(const EprConsts& C, const float* D, const float* P, const float* Ps,
                                float* r, float* RS, int B, cudaStream_t s)
{
    const size_t npix = (size_t)C.nx * C.ny;
    k_sv_split<<<sv_grid(npix, epr_sv_blocks(), B), kSvThreads, 0, s>>>(C, D, P, Ps, r, RS, B);
    epr_count_launch(1);
    return cudaGetLastError();
}

// `part` receives [B][nblk][ns + 1] partials (nblk = epr_sv_blocks(); unused
// blocks of a small map write nothing and are read as the zeros the caller
// leaves there)
cudaError_t epr_launch_sv_update_adj(const EprConsts& C, const float* T, const float* Hs, const float* tb,
                                     float* HB, double* part, int B, float omega, float eps,
                                     float inv_den, cudaStream_t s)
{
    const size_t npix = (size_t)C.nx * C.ny;
    const int nblk = epr_sv_blocks();
    k_sv_update_adj<<<sv_grid(npix, nblk, B), kSvThreads, 0, s>>>(C, T, Hs, tb, HB, part, nblk, B,
                                                                    omega, eps, inv_den);
    epr_count_launch(1);
    return cudaGetLastError();
}

cudaError_t epr_launch_sv_dot(const float* a, const float* b, size_t npix, double* part, int B,
                              cudaStream_t s)
{
    const int nblk = epr_sv_blocks();
    k_sv_dot<<<sv_grid(npix, nblk, B), kSvThreads, 0, s>>>(a, b, npix, part, nblk);
    epr_count_launch(1);
    return cudaGetLastError();
}

cudaError_t epr_launch_sv_splat_field(const EprConsts& C, const float* T, const float* field, float* out,
                                      int line, int B, cudaStream_t s)
{
    const size_t npix = (size_t)C.nx * C.ny;
    k_sv_splat_field<<<sv_grid(npix, 4 * epr_sv_blocks(), B), kSvThreads, 0, s>>>(C, T, field, out, line);
    epr_count_launch(1);
    return cudaGetLastError();
}

// mode 0: the gather's shift term (e = r_s, w = gbar_s); mode 1: the splat's
// (e = Pbar_s, w = I_s).  part: [B][nblk][2].
cudaError_t epr_launch_sv_interp_du(const EprConsts& C, int mode, const float* T, const float* e,
                                    const float* wmap, const float* HB, float* vx, float* vy, float* tn,
                                    double* part, int line, float omega, int B, cudaStream_t s)
{
    const size_t npix = (size_t)C.nx * C.ny;
    const int nblk = epr_sv_blocks();
    const dim3 g = sv_grid(npix, nblk, B);
    if (mode == 0)
        k_sv_interp_du<0><<<g, kSvThreads, 0, s>>>(C, T, e, wmap, HB, vx, vy, tn, part, nblk, line,
                                                    1.f / omega);
    else
        k_sv_interp_du<1><<<g, kSvThreads, 0, s>>>(C, T, e, wmap, HB, vx, vy, tn, part, nblk, line,
                                                    1.f / omega);
    epr_count_launch(1);
    return cudaGetLastError();
}

cudaError_t epr_launch_sv_split_adj(const EprConsts& C, float* RSB, const float* P, const float* Ps,
                                    const float* r, float* Db, int B, cudaStream_t s)
{
    const size_t npix = (size_t)C.nx * C.ny;
    k_sv_split_adj<<<sv_grid(npix, epr_sv_blocks(), B), kSvThreads, 0, s>>>(C, RSB, P, Ps, r, Db, B);
    epr_count_launch(1);
    return cudaGetLastError();
}

cudaError_t epr_launch_sv_gT(const EprConsts& C, const float* vx, const float* vy, float* tn, int B,
                             cudaStream_t s)
{
    k_sv_gT<<<dim3((C.nx + 63) / 64, (C.ny + 3) / 4, B), dim3(64, 4), 0, s>>>(C, vx, vy, tn);
    epr_count_launch(1);
    return cudaGetLastError();
}

// the partials of a producer over maps of npix pixels (sv_grid's block count)
cudaError_t epr_launch_sv_accum(const double* part, size_t npix, int nslot, int slot, double* acc,
                                int nacc, int slot_acc, double scale, int B, cudaStream_t s)
{
    const int nused = (int)sv_grid(npix, epr_sv_blocks(), 1).x;
    k_sv_accum<<<B, 256, 0, s>>>(part, epr_sv_blocks(), nused, nslot, slot, acc, nacc, slot_acc,
                                 scale);
    epr_count_launch(1);
    return cudaGetLastError();
}

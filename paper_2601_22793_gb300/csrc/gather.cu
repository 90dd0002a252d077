// Standalone adjoint of the non-local transport (arXiv 2601.22793, Eq. 4):
// for every object pixel, the bilinear interpolation of a detector map r at
// the pixel's mapped coordinates (x + u_x, y + u_y), u = c_s G[T]; corners
// outside the grid read 0.  This is the exact transpose of the splat.  The
// solver does not use this kernel: it fuses the same gather into the first
// row pass of the preconditioner FFT.
//
// Also: conversion of the splat accumulators to float output maps.
#include "epr_internal.cuh"

namespace {

__device__ __forceinline__ float grad_g(const float* Tb, int y, int x, int ny, int nx, bool along_x)
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

__global__ void k_gather(const EprConsts C, const float* __restrict__ T, const float* __restrict__ r,
                         float* __restrict__ g, int line)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int b = blockIdx.z;
    const int nx = C.nx, ny = C.ny;
    if (x >= nx || y >= ny) return;
    const size_t pb = (size_t)b * nx * ny;
    const float* Tb = T + pb;
    const float* rb = r + pb;
    const float cs = C.xt ? xt_get(C, EPR_XT_C, line, x) : C.c[line];
    const float lim = 2.f * (float)(nx > ny ? nx : ny);
    const float ux = fminf(fmaxf(cs * grad_g(Tb, y, x, ny, nx, true), -lim), lim);
    const float uy = fminf(fmaxf(cs * grad_g(Tb, y, x, ny, nx, false), -lim), lim);
    const float fx = floorf(ux), fy = floorf(uy);
    const float dx = ux - fx, dy = uy - fy;
    const int cx = x + (int)fx, cy = y + (int)fy;
    float acc = 0.f;
    const bool x0 = cx >= 0 && cx < nx, x1 = cx + 1 >= 0 && cx + 1 < nx;
    if (cy >= 0 && cy < ny) {
        const size_t row = (size_t)cy * nx;
        if (x0) acc += (1.f - dx) * (1.f - dy) * __ldg(&rb[row + cx]);
        if (x1) acc += dx * (1.f - dy) * __ldg(&rb[row + cx + 1]);
    }
    if (cy + 1 >= 0 && cy + 1 < ny) {
        const size_t row = (size_t)(cy + 1) * nx;
        if (x0) acc += (1.f - dx) * dy * __ldg(&rb[row + cx]);
        if (x1) acc += dx * dy * __ldg(&rb[row + cx + 1]);
    }
    g[pb + (size_t)y * nx + x] = acc;
}

__global__ void k_fx_to_float(const unsigned long long* __restrict__ q, float* __restrict__ out, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = (float)q[i] * EPR_FX_INV;
}

}  // namespace

cudaError_t epr_launch_gather(const EprConsts& C, const float* T, const float* r, float* g, int line,
                              int batch, cudaStream_t stream)
{
    dim3 blk(64, 4);
    dim3 grid((C.nx + 63) / 64, (C.ny + 3) / 4, batch);
    k_gather<<<grid, blk, 0, stream>>>(C, T, r, g, line);
    epr_count_launch(1);
    return cudaGetLastError();
}

cudaError_t epr_launch_fx_to_float(const unsigned long long* q, float* out, size_t n, cudaStream_t stream)
{
    const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    k_fx_to_float<<<blocks > 0 ? blocks : 1, 256, 0, stream>>>(q, out, n);
    epr_count_launch(1);
    return cudaGetLastError();
}

// Forward non-local transport: the conservative bilinear redistribution of
// the object intensity of every spectral line onto the detector grid
// (arXiv 2601.22793, Eq. 3 and "Discrete implementation: conservative
// bilinear redistribution"), with the polychromatic sum of Eq. 5.
//
// Design (destination-tile binning):
//  * A block owns one TH x TW destination tile of one projection and holds
//    its accumulators (one per line) in shared memory.
//  * It scans every source pixel whose shifted corners can land in the tile:
//    the tile grown by R = smax + 1 pixels on each side.  The thickness of
//    that region plus a one-pixel ring (for the gradient) is staged in shared
//    memory with coalesced loads.
//  * Per source and line it forms the shift u = c_s G[T] (central
//    differences, one-sided at the grid edges), splits u into floor and
//    fraction (the integer pixel index never passes through float), and adds
//    f_s exp(-mu_s T) times the four bilinear weights to the corners inside
//    the tile with shared-memory atomics.  exp is evaluated only when the
//    source reaches the tile.
//  * Every destination pixel is written exactly once, with plain coalesced
//    stores: no zero fill and no global atomics on the fast path.
//  * A source-line with |u| > smax in either axis is never splatted by the
//    scan; the block that owns the source pixel appends it (with a bit mask
//    of its long lines) to a per-projection overflow list.  The last block of
//    the projection to finish (arrival counter after a memory fence) adds
//    those contributions with global atomics, so no mass is lost whatever
//    the shift.
//  * Fixed-point mode accumulates round(v * 2^40) in uint64 (all
//    contributions are non-negative) in shared and global memory: integer
//    addition is associative, so the result is bit-identical across runs.
#include "epr_internal.cuh"

namespace {

constexpr int kSplatThreads = 256;

struct SplatArgs {
    const float* T;          // [B][ny][nx]
    float* P;                // [B][ny][nx]          (float mode)
    float* Ps;               // [B][ns][ny][nx] or NULL (float mode, ns > 1)
    unsigned long long* Pq;  // fixed-point mode
    unsigned long long* Psq;
    int* ovf_idx;
    unsigned int* ovf_mask;
    EprProjState* st;
    unsigned int* err;
    int TH, TW, tiles_x, tiles_y;
    int check_done;
};

// numpy.gradient semantics along one axis from three neighbours.
__device__ __forceinline__ float grad1(float lo, float mid, float hi, int i, int n)
{
    if (i == 0) return hi - mid;
    if (i == n - 1) return mid - lo;
    return 0.5f * (hi - lo);
}

template <bool DET>
__device__ __forceinline__ void acc_add(void* acc, int idx, float v)
{
    if constexpr (DET) {
        unsigned long long q = (unsigned long long)__float2ll_rn(v * EPR_FX_SCALE);
        atomicAdd(reinterpret_cast<unsigned long long*>(acc) + idx, q);
    } else {
        atomicAdd(reinterpret_cast<float*>(acc) + idx, v);
    }
}

template <bool DET>
__global__ void __launch_bounds__(kSplatThreads)
k_splat(const EprConsts C, const SplatArgs A)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int b = blockIdx.z;
    if (A.check_done && A.st[b].done) return;
    const int nx = C.nx, ny = C.ny, ns = C.ns;
    const int TH = A.TH, TW = A.TW;
    const int ty0 = blockIdx.y * TH, tx0 = blockIdx.x * TW;
    const int R = C.smax + 1;
    const int RH = TH + 2 * R, RW = TW + 2 * R;     // source region
    const int SH = RH + 2, SW = RW + 2;              // staged thickness
    const int tile = TH * TW;
    const size_t npix = (size_t)nx * ny;

    // shared layout: accumulators [ns][TH][TW], then thickness [SH][SW]
    void* acc = smem;
    const size_t acc_bytes = (size_t)ns * tile * (DET ? 8 : 4);
    float* Ts = reinterpret_cast<float*>(smem + ((acc_bytes + 15) & ~size_t(15)));
    const float* Tb = A.T + (size_t)b * npix;

    // stage thickness rows ty0-R-1 .. ty0+TH+R and cols tx0-R-1 .. tx0+TW+R
    const int sy0 = ty0 - R - 1, sx0 = tx0 - R - 1;
    for (int i = threadIdx.x; i < SH * SW; i += kSplatThreads) {
        const int ly = i / SW, lx = i - ly * SW;
        const int gy = sy0 + ly, gx = sx0 + lx;
        float v = 0.f;
        if (gy >= 0 && gy < ny && gx >= 0 && gx < nx) v = __ldg(&Tb[(size_t)gy * nx + gx]);
        Ts[i] = v;
    }
    if constexpr (DET) {
        unsigned long long* a = reinterpret_cast<unsigned long long*>(acc);
        for (int i = threadIdx.x; i < ns * tile; i += kSplatThreads) a[i] = 0ull;
    } else {
        float* a = reinterpret_cast<float*>(acc);
        for (int i = threadIdx.x; i < ns * tile; i += kSplatThreads) a[i] = 0.f;
    }
    __syncthreads();

    const float fsmax = (float)C.smax;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int ly = warp; ly < RH; ly += kSplatThreads / 32) {
        const int sy = ty0 - R + ly;
        if (sy < 0 || sy >= ny) continue;
        for (int lx = lane; lx < RW; lx += 32) {
            const int sx = tx0 - R + lx;
            if (sx < 0 || sx >= nx) continue;
            const float* tp = Ts + (ly + 1) * SW + (lx + 1);
            const float t = tp[0];
            const float gx = grad1(tp[-1], t, tp[1], sx, nx);
            const float gy = grad1(tp[-SW], t, tp[SW], sy, ny);
            const bool own = (ly >= R) && (ly < R + TH) && (lx >= R) && (lx < R + TW);
            unsigned int far = 0u;
            for (int s = 0; s < ns; ++s) {
                const float ux = C.c[s] * gx, uy = C.c[s] * gy;
                if (!(fabsf(ux) <= fsmax && fabsf(uy) <= fsmax)) {
                    far |= 1u << s;
                    continue;
                }
                const float fx = floorf(ux), fy = floorf(uy);
                const float dx = ux - fx, dy = uy - fy;
                const int cx = sx + (int)fx - tx0, cy = sy + (int)fy - ty0;  // corner 00, tile-local
                if (cx < -1 || cx >= TW || cy < -1 || cy >= TH) continue;
                const float m = C.f[s] * __expf(-C.mu[s] * t);
                const float w00 = (1.f - dx) * (1.f - dy), w10 = dx * (1.f - dy);
                const float w01 = (1.f - dx) * dy, w11 = dx * dy;
                const int base = s * tile;
                const bool x0in = cx >= 0, x1in = cx + 1 < TW;
                const bool y0in = cy >= 0, y1in = cy + 1 < TH;
                if (y0in && x0in) acc_add<DET>(acc, base + cy * TW + cx, m * w00);
                if (y0in && x1in) acc_add<DET>(acc, base + cy * TW + cx + 1, m * w10);
                if (y1in && x0in) acc_add<DET>(acc, base + (cy + 1) * TW + cx, m * w01);
                if (y1in && x1in) acc_add<DET>(acc, base + (cy + 1) * TW + cx + 1, m * w11);
            }
            if (far && own) {
                const int pos = atomicAdd(&A.st[b].ovf_count, 1);
                if (pos < C.ovf_cap) {
                    A.ovf_idx[(size_t)b * C.ovf_cap + pos] = sy * nx + sx;
                    A.ovf_mask[(size_t)b * C.ovf_cap + pos] = far;
                } else {
                    atomicOr(A.err, EPR_DEVERR_OVERFLOW);
                }
            }
        }
    }
    __syncthreads();

    // flush: every pixel of the tile inside the grid, once, coalesced
    for (int i = threadIdx.x; i < tile; i += kSplatThreads) {
        const int ly = i / TW, lx = i - ly * TW;
        const int gy = ty0 + ly, gx = tx0 + lx;
        if (gy >= ny || gx >= nx) continue;
        const size_t o = (size_t)gy * nx + gx;
        if constexpr (DET) {
            const unsigned long long* a = reinterpret_cast<const unsigned long long*>(acc);
            unsigned long long sum = 0ull;
            for (int s = 0; s < ns; ++s) {
                const unsigned long long q = a[s * tile + i];
                sum += q;
                if (ns > 1) A.Psq[((size_t)b * ns + s) * npix + o] = q;
            }
            A.Pq[(size_t)b * npix + o] = sum;
        } else {
            const float* a = reinterpret_cast<const float*>(acc);
            float sum = 0.f;
            for (int s = 0; s < ns; ++s) {
                const float q = a[s * tile + i];
                sum += q;
                if (ns > 1) A.Ps[((size_t)b * ns + s) * npix + o] = q;
            }
            A.P[(size_t)b * npix + o] = sum;
        }
    }

    // last block of this projection adds the overflow list
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int nblk = (unsigned int)(A.tiles_x * A.tiles_y);
        const unsigned int prev = atomicAdd(&A.st[b].cnt_splat, 1u);
        s_last = (prev == nblk - 1u);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int cnt_raw = *((volatile int*)&A.st[b].ovf_count);
    const int cnt = cnt_raw < C.ovf_cap ? cnt_raw : C.ovf_cap;
    for (int e = threadIdx.x; e < cnt; e += kSplatThreads) {
        const int pix = A.ovf_idx[(size_t)b * C.ovf_cap + e];
        const unsigned int mask = A.ovf_mask[(size_t)b * C.ovf_cap + e];
        const int sy = pix / nx, sx = pix - sy * nx;
        const float* tp = Tb + pix;
        const float t = tp[0];
        const float gx = grad1(sx > 0 ? tp[-1] : t, t, sx < nx - 1 ? tp[1] : t, sx, nx);
        const float gy = grad1(sy > 0 ? tp[-nx] : t, t, sy < ny - 1 ? tp[nx] : t, sy, ny);
        for (int s = 0; s < ns; ++s) {
            if (!((mask >> s) & 1u)) continue;
            const float ux = C.c[s] * gx, uy = C.c[s] * gy;
            const float fx = floorf(ux), fy = floorf(uy);
            const float dx = ux - fx, dy = uy - fy;
            const float m = C.f[s] * __expf(-C.mu[s] * t);
            const float w[4] = {(1.f - dx) * (1.f - dy), dx * (1.f - dy), (1.f - dx) * dy, dx * dy};
            // corner coordinates in float first: a huge shift must not wrap an int
            const float cxf = (float)sx + fx, cyf = (float)sy + fy;
            for (int k = 0; k < 4; ++k) {
                const float xf = cxf + (float)(k & 1), yf = cyf + (float)(k >> 1);
                if (!(xf >= 0.f && xf < (float)nx && yf >= 0.f && yf < (float)ny)) continue;
                const size_t o = (size_t)(int)yf * nx + (int)xf;
                const float v = m * w[k];
                if constexpr (DET) {
                    const unsigned long long q = (unsigned long long)__float2ll_rn(v * EPR_FX_SCALE);
                    atomicAdd(&A.Pq[(size_t)b * npix + o], q);
                    if (ns > 1) atomicAdd(&A.Psq[((size_t)b * ns + s) * npix + o], q);
                } else {
                    atomicAdd(&A.P[(size_t)b * npix + o], v);
                    if (ns > 1) atomicAdd(&A.Ps[((size_t)b * ns + s) * npix + o], v);
                }
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (cnt > 0) A.st[b].ovf_total += cnt;
        A.st[b].ovf_count = 0;
        A.st[b].cnt_splat = 0u;
        __threadfence();
    }
}

}  // namespace

// Host launcher.  TH x TW is the destination tile; shared memory =
// ns * TH * TW accumulators + (TH + 2R + 2)(TW + 2R + 2) floats.
cudaError_t epr_launch_splat(const EprConsts& C, const EprWork& W, const float* T, int batch,
                             int TH, int TW, int check_done, cudaStream_t stream)
{
    SplatArgs A;
    A.T = T;
    A.P = W.P;
    A.Ps = W.Ps;
    A.Pq = W.Pq;
    A.Psq = W.Psq;
    A.ovf_idx = W.ovf_idx;
    A.ovf_mask = W.ovf_mask;
    A.st = W.st;
    A.err = W.err;
    A.TH = TH;
    A.TW = TW;
    A.tiles_x = (C.nx + TW - 1) / TW;
    A.tiles_y = (C.ny + TH - 1) / TH;
    A.check_done = check_done;
    const int R = C.smax + 1;
    const size_t acc_bytes = (size_t)C.ns * TH * TW * (C.det ? 8 : 4);
    const size_t smem = ((acc_bytes + 15) & ~size_t(15)) +
                        (size_t)(TH + 2 * R + 2) * (TW + 2 * R + 2) * sizeof(float);
    dim3 grid(A.tiles_x, A.tiles_y, batch);
    if (C.det) k_splat<true><<<grid, kSplatThreads, smem, stream>>>(C, A);
    else k_splat<false><<<grid, kSplatThreads, smem, stream>>>(C, A);
    epr_count_launch(1);
    return cudaGetLastError();
}

size_t epr_splat_smem(const EprConsts& C, int TH, int TW)
{
    const int R = C.smax + 1;
    const size_t acc_bytes = (size_t)C.ns * TH * TW * (C.det ? 8 : 4);
    return ((acc_bytes + 15) & ~size_t(15)) + (size_t)(TH + 2 * R + 2) * (TW + 2 * R + 2) * sizeof(float);
}

cudaError_t epr_splat_init()
{
    cudaError_t e = epr_allow_max_smem(k_splat<true>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_splat<false>);
    return e;
}

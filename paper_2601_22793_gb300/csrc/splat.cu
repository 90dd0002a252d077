// Forward non-local transport: the conservative bilinear redistribution of
// the object intensity of every spectral line onto the detector grid
// (arXiv 2601.22793, Eq. 3 and "Discrete implementation: conservative
// bilinear redistribution"), with the polychromatic sum of Eq. 5.
//
// Design (destination-tile binning):
//  * A block owns one TH x TW destination tile of one projection and holds
//    its accumulators (one per line) in shared memory.
//  * It scans every source pixel whose shifted corners can land in the tile:
//    the tile grown by R = reach + 1 pixels on each side.  The thickness of
//    that region plus a one-pixel ring (for the gradient) is staged in shared
//    memory with coalesced loads.  Blocks whose staged region lies inside the
//    grid take a path without edge tests.
//  * Per source and line it forms the shift u = c_s G[T] (central
//    differences, one-sided at the grid edges), splits u into floor and
//    fraction (the integer pixel index never passes through float), and adds
//    f_s exp(-mu_s T) times the four bilinear weights to the corners inside
//    the tile with shared-memory atomics.  exp is evaluated only when the
//    source reaches the tile.
//  * The shared accumulators are integers, because integer shared-memory
//    atomics are single instructions while float ones are not.  The float
//    mode adds round(v * 2^S) in uint32 with S chosen from the reach so that
//    no pixel can overflow: at most (2 reach + 3)^2 sources reach a pixel,
//    each with a contribution <= f_s <= 1, so 2^(32-S) >= (2 reach + 3)^2.
//    With a factor 2 of headroom, 2^(32-S) >= 2 (2 reach + 3)^2 holds for
//    contributions up to 2 f_s, and a source whose intensity exceeds that
//    (T < -ln 2 / mu_s, a negative thickness far outside any physical
//    iterate) takes the overflow path with the long shifts.  For reach 4,
//    S = 24: a rounding error of at most 3e-8 per contribution, half an fp32
//    ulp of a unit intensity.
//  * Every destination pixel is written exactly once, with plain coalesced
//    stores: no zero fill and no global atomics on the fast path.  In the
//    monochromatic float solve the flush stores the residual D - P instead
//    of P (the adjoint gather then reads one value per corner).
//  * A source-line with |u| > reach in either axis (or T below the bound
//    above) is never splatted by the scan; the block that owns the source
//    pixel appends it (with a bit mask of its long lines, its thickness and
//    twice its gradient) to a per-projection overflow list, and a second
//    kernel adds those contributions with global atomics.  No mass is lost,
//    whatever the shift.  The list fill counter alternates between two slots
//    by iteration parity, so the overflow kernel can clear the next slot.
//  * Fixed-point mode accumulates round(v * 2^40) in uint64 (contributions
//    are non-negative) in shared and global memory: integer addition is
//    associative, so the result is bit-identical across runs.
#include <type_traits>

#include "epr_internal.cuh"

namespace {

// Threads of a splat block: 256 for one line; 512 for several lines (a
// runtime count, or 4 or 8 at compile time), whose per-line accumulators
// limit a 32 x 64 tile to two blocks per SM: the wider block doubles the
// warps that hide the latency of the shared-memory atomics.  With the line
// count known at compile time the line loop unrolls, so the compiler can
// interleave the lines' dependency chains.
__host__ __device__ constexpr int splat_threads(int NS) { return NS == 1 ? 256 : 512; }

struct SplatArgs {
    const float* T;          // [B][ny][nx]
    const float* D;          // [B][ny][nx] (residual output)
    float* P;                // [B][ny][nx]   P, or D - P (residual output)
    float* Ps;               // [B][ns][ny][nx] or NULL (float mode, ns > 1)
    unsigned long long* Pq;  // fixed-point mode
    unsigned long long* Psq;
    int* ovf_idx;
    unsigned int* ovf_mask;
    float4* ovf_tg;          // (T, twice the gradient x, y, 0) of each entry
    EprProjState* st;
    unsigned int* err;
    int parity;
    int check_done;
    float fxs, fxs_inv;      // float mode: scale 2^S of the uint32 accumulators
};

// numpy.gradient semantics along one axis from three neighbours.
__device__ __forceinline__ float grad1(float lo, float mid, float hi, int i, int n)
{
    if (i == 0) return hi - mid;
    if (i == n - 1) return mid - lo;
    return 0.5f * (hi - lo);
}

// i / d for 0 <= i < 2^20 and d < 2^12 without an integer division
__device__ __forceinline__ int fdiv(int i, float inv_d) { return (int)(((float)i + 0.5f) * inv_d); }

// v is already scaled by the accumulator's 2^S
template <bool DET>
__device__ __forceinline__ void acc_add(void* acc, int idx, float v)
{
    if constexpr (DET) {
        unsigned long long q = (unsigned long long)__float2ll_rn(v);
        atomicAdd(reinterpret_cast<unsigned long long*>(acc) + idx, q);
    } else {
        atomicAdd(reinterpret_cast<unsigned int*>(acc) + idx, __float2uint_rn(v));
    }
}

// NS = 1: single line known at compile time; NS = 0: C.ns lines.
// Shared layout: accumulators [ns][TH + 2][TW + 2]; the staged thickness window
// [SH][SWa] whose first column ax0 = tx0 - HX is 16-byte aligned (HX = R + 1
// rounded up to 4) so rows load as float4; a list of far sources.
constexpr int kFarList = 256;
constexpr int kQuad = 4;   // sources per scan work item

// The tile shape is a compile-time parameter (64 x 64, 32 x 64, 64 x 32 or
// 32 x 32, chosen on the host), and so is the reach RC of the float solves
// for the reaches the tuner tries (3, 4, 6; RC = 0 takes C.smax), so every
// tile- and reach-derived index, stride and offset folds into immediates.
// Five blocks per SM (48 registers; a 64 x 64 tile at reach 4 takes 44 KB of
// shared memory); the mono residual kernel with a runtime reach needs more
// registers and runs four.
// XT: an x-dependent spectrum, the line constants read per source column
// from the plan's table (runtime line count and reach only).
// OCC > 0: that many blocks per SM (six for the one-line residual kernels of
// the tiles smaller than 64 x 64 at reach 3 and 4: 40 registers, no spills).
template <int NS, bool DET, bool RESID, int TH, int TW, int RC = 0, bool XT = false, int OCC = 0>
__global__ void __launch_bounds__(splat_threads(NS),
                                  OCC > 0 ? OCC : NS != 1 ? 2 : ((RESID && RC == 0) ? 4 : 5))
k_splat(const EprConsts C, const SplatArgs A)
{
    constexpr int kSplatThreads = splat_threads(NS);
    static_assert((TW & (TW - 1)) == 0 && TH * TW <= 4 * 4 * kSplatThreads, "tile shape");
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_far_idx[kFarList];
    __shared__ unsigned int s_far_mask[kFarList];
    __shared__ int s_far_n, s_far_base;
    const int b = blockIdx.z;
    const int nx = C.nx, ny = C.ny;
    const int ns = NS ? NS : C.ns;
    const int ty0 = blockIdx.y * TH, tx0 = blockIdx.x * TW;
    const int smax = RC > 0 ? RC : C.smax;
    const int R = smax + 1;
    const int RH = TH + 2 * R, RW = TW + 2 * R;     // source region
    const int RHq = (RH + kQuad - 1) / kQuad;         // its rows in quads
    const int HX = (R + 1 + 3) & ~3;
    const int SH = RHq * kQuad + 2, SWa = TW + 2 * HX;   // staged thickness
    const int coff = HX - R - 1;                     // staged column of source column tx0 - R - 1
    constexpr int tile = TH * TW;
    // accumulators [ns][TH + 2][TW + 2]: the tile with a one-pixel apron, so
    // the four corners of any source that touches the tile have a slot
    constexpr int AP = TW + 2, ACC = (TH + 2) * AP;
    const size_t npix = (size_t)nx * ny;
    const int tid = threadIdx.x;

    void* acc = smem;
    const size_t acc_bytes = (size_t)ns * ACC * (DET ? 8 : 4);
    float* Ts = reinterpret_cast<float*>(smem + ((acc_bytes + 15) & ~size_t(15)));
    const float* Tb = A.T + (size_t)b * npix;
    if (tid == 0) s_far_n = 0;

    // the detector data of the tile, fetched before the scan (residual output)
    constexpr int kDq = 4;   // float4 per thread: tiles up to 64 x 64
    float4 dreg[kDq];
    constexpr int nq = tile >> 2;
    constexpr int tw4 = TW >> 2;
    if constexpr (RESID) {
#pragma unroll
        for (int k = 0; k < kDq; ++k) {
            const int i4 = tid + k * kSplatThreads;
            dreg[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (i4 < nq) {
                const int ly = i4 / tw4, lx = (i4 - ly * tw4) << 2;
                const int gy = ty0 + ly, gx = tx0 + lx;
                if (gy < ny && gx < nx)
                    dreg[k] = __ldg(reinterpret_cast<const float4*>(A.D + (size_t)b * npix + (size_t)gy * nx + gx));
            }
        }
    }

    if constexpr (DET) {
        unsigned long long* a = reinterpret_cast<unsigned long long*>(acc);
        for (int i = tid; i < ns * ACC; i += kSplatThreads) a[i] = 0ull;
    } else {   // ACC = 4 (TH/2 + 1)(TW/2 + 1)
        uint4* a = reinterpret_cast<uint4*>(acc);
        for (int i = tid; i < ns * ACC / 4; i += kSplatThreads) a[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    // T, the done flags and the overflow counters come from earlier kernels
    epr_grid_wait();
    if (A.check_done && A.st[b].done) return;

    const int sy0 = ty0 - R - 1, sx0 = tx0 - R - 1, ax0 = tx0 - HX;
    const bool interior = sy0 >= 0 && sx0 >= 0 && sy0 + SH <= ny && sx0 + RW + 2 <= nx;
    {
        const int q = SWa >> 2;
        const float inv_q = 1.f / (float)q;
        for (int i = tid; i < SH * q; i += kSplatThreads) {
            const int ly = fdiv(i, inv_q), c4 = i - ly * q;
            const int gy = sy0 + ly, gx = ax0 + 4 * c4;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (gy >= 0 && gy < ny && gx >= 0 && gx < nx)   // nx % 4 == 0: all four or none
                v = __ldg(reinterpret_cast<const float4*>(Tb + (size_t)gy * nx + gx));
            reinterpret_cast<float4*>(Ts)[i] = v;
        }
    }
    __syncthreads();

    const float fsmax = (float)smax;
    // the accumulator scale 2^S is folded into the line weight: a power of two
    // scales exactly, so each contribution rounds to the same integer
    const float fxs = DET ? EPR_FX_SCALE : A.fxs;
    // One source at tile-local (ly, lx) with thickness t and twice its
    // gradient: every line's shift, contributions and far flag.  Gradients
    // are kept doubled (hi - lo), and half the shift constant multiplies
    // them: 0.5 scales exactly, so u is the same float.
    auto source = [&](int ly, int lx, float t, float gx2, float gy2) {
        unsigned int far = 0u;
        const int sxc = XT ? tx0 - R + lx : 0;   // source column (inside the grid)
#pragma unroll(NS ? NS : 1)
        for (int s = 0; s < ns; ++s) {
            const float ch = 0.5f * (XT ? xt_get(C, EPR_XT_C, s, sxc) : C.c[s]);
            const float ux = ch * gx2, uy = ch * gy2;
            const float tneg = XT ? xt_get(C, EPR_XT_TNEG, s, sxc) : C.tneg[s];
            if (fabsf(ux) <= fsmax && fabsf(uy) <= fsmax && t >= tneg) {
                const float fx = floorf(ux), fy = floorf(uy);
                const int cx = lx - R + (int)fx, cy = ly - R + (int)fy;  // corner 00, tile-local
                // all four corners have a slot (apron) when one is in the tile
                if ((unsigned)(cx + 1) <= (unsigned)TW && (unsigned)(cy + 1) <= (unsigned)TH) {
                    const float dx = ux - fx, dy = uy - fy;
                    const float fs = XT ? xt_get(C, EPR_XT_F, s, sxc) : C.f[s];
                    const float mus = XT ? xt_get(C, EPR_XT_MU, s, sxc) : C.mu[s];
                    const float m = (fs * fxs) * __expf(-mus * t);   // 2^S f e^(-mu t)
                    const float mx1 = m * dx, mx0 = m - mx1;          // m (1 - dx), m dx
                    const float w = 1.f - dy;
                    const int idx = s * ACC + (cy + 1) * AP + (cx + 1);
                    acc_add<DET>(acc, idx, mx0 * w);
                    acc_add<DET>(acc, idx + 1, mx1 * w);
                    acc_add<DET>(acc, idx + AP, mx0 * dy);
                    acc_add<DET>(acc, idx + AP + 1, mx1 * dy);
                }
            } else {
                far |= 1u << s;
            }
        }
        if (far && (unsigned)(ly - R) < (unsigned)TH && (unsigned)(lx - R) < (unsigned)TW) {
            const int sy = ty0 - R + ly, sx = tx0 - R + lx;
            const int pos = atomicAdd(&s_far_n, 1);
            if (pos < kFarList) {
                s_far_idx[pos] = sy * nx + sx;
                s_far_mask[pos] = far;
            } else {   // list full: append to the global list directly
                const int gpos = atomicAdd(&A.st[b].ovf_count[A.parity], 1);
                if (gpos < C.ovf_cap) {
                    A.ovf_idx[(size_t)b * C.ovf_cap + gpos] = sy * nx + sx;
                    A.ovf_mask[(size_t)b * C.ovf_cap + gpos] = far;
                    A.ovf_tg[(size_t)b * C.ovf_cap + gpos] = make_float4(t, gx2, gy2, 0.f);
                } else {
                    atomicOr(A.err, EPR_DEVERR_OVERFLOW);
                }
            }
        }
    };
    // The scan: a thread takes kQuad vertically adjacent sources of one
    // column (rows ly0 .. ly0 + kQuad - 1 of the region, padded to a multiple
    // of kQuad; padding rows cannot reach the tile and are not owned by it),
    // reusing the column's thickness values.  Specialised for blocks whose
    // staged region lies inside the grid (central differences everywhere, no
    // edge tests) and for edge blocks.  Work item (qy, lx) is advanced by
    // kSplatThreads = dly quad rows + dlx columns.
    const int nitem = RHq * RW;
    const int dly = kSplatThreads / RW, dlx = kSplatThreads - dly * RW;
    auto scan = [&](auto interior_tag) {
        constexpr bool IN = decltype(interior_tag)::value;
        int qy = tid / RW, lx = tid - (tid / RW) * RW;
        for (int i = tid; i < nitem; i += kSplatThreads, lx += dlx,
                 qy += dly + (lx >= RW ? 1 : 0), lx -= (lx >= RW ? RW : 0)) {
            const int ly0 = qy * kQuad;
            const float* tp = Ts + (ly0 + 1) * SWa + (lx + 1 + coff);   // source (ly0, lx)
            float col[kQuad + 2];   // the column, rows ly0 - 1 .. ly0 + kQuad
#pragma unroll
            for (int j = 0; j < kQuad + 2; ++j) col[j] = tp[(j - 1) * SWa];
#pragma unroll
            for (int j = 0; j < kQuad; ++j) {
                const float t = col[j + 1];
                float gx2, gy2;   // twice the gradient
                if constexpr (IN) {
                    gx2 = tp[j * SWa + 1] - tp[j * SWa - 1];
                    gy2 = col[j + 2] - col[j];
                } else {
                    const int sy = ty0 - R + ly0 + j, sx = tx0 - R + lx;
                    if (sy < 0 || sy >= ny || sx < 0 || sx >= nx) continue;
                    gx2 = 2.f * grad1(tp[j * SWa - 1], t, tp[j * SWa + 1], sx, nx);
                    gy2 = 2.f * grad1(col[j], t, col[j + 2], sy, ny);
                }
                source(ly0 + j, lx, t, gx2, gy2);
            }
        }
    };
    if (interior) scan(std::true_type{});
    else scan(std::false_type{});
    __syncthreads();
    epr_grid_release();

    // far sources of this block: one reservation in the global list.  Each
    // entry carries T and twice the gradient, formed from the staged window
    // as in the scan (the same bits), so the overflow kernel reads no T.
    const int nfar = s_far_n < kFarList ? s_far_n : kFarList;
    if (nfar > 0) {
        if (tid == 0) s_far_base = atomicAdd(&A.st[b].ovf_count[A.parity], nfar);
        __syncthreads();
        for (int e = tid; e < nfar; e += kSplatThreads) {
            const int gpos = s_far_base + e;
            if (gpos < C.ovf_cap) {
                const int pix = s_far_idx[e];
                const int sy = pix / nx, sx = pix - sy * nx;
                const int ly = sy - ty0 + R, lx = sx - tx0 + R;   // in the source region
                const float* tp = Ts + (ly + 1) * SWa + (lx + 1 + coff);
                const float t = tp[0];
                float gx2, gy2;
                if (interior) {
                    gx2 = tp[1] - tp[-1];
                    gy2 = tp[SWa] - tp[-SWa];
                } else {
                    gx2 = 2.f * grad1(tp[-1], t, tp[1], sx, nx);
                    gy2 = 2.f * grad1(tp[-SWa], t, tp[SWa], sy, ny);
                }
                A.ovf_idx[(size_t)b * C.ovf_cap + gpos] = pix;
                A.ovf_mask[(size_t)b * C.ovf_cap + gpos] = s_far_mask[e];
                A.ovf_tg[(size_t)b * C.ovf_cap + gpos] = make_float4(t, gx2, gy2, 0.f);
            } else {
                atomicOr(A.err, EPR_DEVERR_OVERFLOW);
            }
        }
    }

    // flush: every pixel of the tile inside the grid, once, coalesced
    if constexpr (RESID) {
        const unsigned int* a = reinterpret_cast<const unsigned int*>(acc);
        const float inv = A.fxs_inv;
#pragma unroll
        for (int k = 0; k < kDq; ++k) {
            const int i4 = tid + k * kSplatThreads;
            if (i4 >= nq) continue;
            const int ly = i4 / tw4, lx = (i4 - ly * tw4) << 2;
            const int gy = ty0 + ly, gx = tx0 + lx;
            if (gy >= ny || gx >= nx) continue;
            const unsigned int* v = a + (ly + 1) * AP + lx + 1;
            const float4 d = dreg[k];
            *reinterpret_cast<float4*>(A.P + (size_t)b * npix + (size_t)gy * nx + gx) =
                make_float4(d.x - (float)v[0] * inv, d.y - (float)v[1] * inv,
                            d.z - (float)v[2] * inv, d.w - (float)v[3] * inv);
        }
    } else {
        for (int i = tid; i < tile; i += kSplatThreads) {
            const int ly = i / TW, lx = i & (TW - 1);
            const int gy = ty0 + ly, gx = tx0 + lx;
            if (gy >= ny || gx >= nx) continue;
            const size_t o = (size_t)b * npix + (size_t)gy * nx + gx;
            if constexpr (DET) {
                const unsigned long long* a = reinterpret_cast<const unsigned long long*>(acc);
                unsigned long long sum = 0ull;
                for (int s = 0; s < ns; ++s) {
                    const unsigned long long q = a[s * ACC + (ly + 1) * AP + lx + 1];
                    sum += q;
                    if (ns > 1) A.Psq[(size_t)s * npix + o + (size_t)b * (ns - 1) * npix] = q;
                }
                A.Pq[o] = sum;
            } else {
                // sum <= 2 (2 reach + 3)^2 sum_s f_s: no overflow either
                const unsigned int* a = reinterpret_cast<const unsigned int*>(acc);
                unsigned int sum = 0u;
                for (int s = 0; s < ns; ++s) {
                    const unsigned int q = a[s * ACC + (ly + 1) * AP + lx + 1];
                    sum += q;
                    if (ns > 1)
                        A.Ps[(size_t)s * npix + o + (size_t)b * (ns - 1) * npix] = (float)q * A.fxs_inv;
                }
                A.P[o] = (float)sum * A.fxs_inv;
            }
        }
    }
}

// The long-shift sources of the overflow list, added with global atomics.
template <bool DET, bool RESID, bool XT = false>
__global__ void __launch_bounds__(128) k_splat_overflow(const EprConsts C, const SplatArgs A)
{
    const int b = blockIdx.y;
    epr_grid_wait();
    if (A.check_done && A.st[b].done) return;
    epr_grid_release();
    const int nx = C.nx, ny = C.ny, ns = C.ns;
    const size_t npix = (size_t)nx * ny;
    const int cnt_raw = A.st[b].ovf_count[A.parity];
    const int cnt = cnt_raw < C.ovf_cap ? cnt_raw : C.ovf_cap;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        A.st[b].ovf_count[A.parity ^ 1] = 0;   // the next splat's slot
        if (cnt > 0) A.st[b].ovf_total += cnt;
    }
    // entries come with T and twice the gradient; the first round's entry is
    // loaded together with the count (every slot below the capacity exists)
    const int stride = gridDim.x * blockDim.x;
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    int pix = 0;
    unsigned int mask = 0u;
    float4 tg = make_float4(0.f, 0.f, 0.f, 0.f);
    if (e < C.ovf_cap) {
        pix = A.ovf_idx[(size_t)b * C.ovf_cap + e];
        mask = A.ovf_mask[(size_t)b * C.ovf_cap + e];
        tg = A.ovf_tg[(size_t)b * C.ovf_cap + e];
    }
    for (; e < cnt; e += stride) {
        if (e >= stride) {   // later rounds
            pix = A.ovf_idx[(size_t)b * C.ovf_cap + e];
            mask = A.ovf_mask[(size_t)b * C.ovf_cap + e];
            tg = A.ovf_tg[(size_t)b * C.ovf_cap + e];
        }
        const int sy = pix / nx, sx = pix - sy * nx;
        const float t = tg.x;
        for (int s = 0; s < ns; ++s) {
            if (!((mask >> s) & 1u)) continue;
            const float ch = 0.5f * (XT ? xt_get(C, EPR_XT_C, s, sx) : C.c[s]);
            const float ux = ch * tg.y, uy = ch * tg.z;
            const float fx = floorf(ux), fy = floorf(uy);
            const float dx = ux - fx, dy = uy - fy;
            const float fs = XT ? xt_get(C, EPR_XT_F, s, sx) : C.f[s];
            const float mus = XT ? xt_get(C, EPR_XT_MU, s, sx) : C.mu[s];
            const float m = fs * __expf(-mus * t);
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
                } else if constexpr (RESID) {
                    atomicAdd(&A.P[(size_t)b * npix + o], -v);
                } else {
                    atomicAdd(&A.P[(size_t)b * npix + o], v);
                    if (ns > 1) atomicAdd(&A.Ps[((size_t)b * ns + s) * npix + o], v);
                }
            }
        }
    }
}

// The residual and its split over the lines (the weights P_s / P of the
// "Iteration structure"; r f_s where P vanishes), once per pixel after the
// overflow sources are in: P <- D - P and P_s <- (D - P) P_s / P as float
// maps, so that the adjoint gather reads one value per corner and line.  In
// fixed-point mode the sums are read from the integer maps.
// The float mode takes four pixels per thread and loads every line's P_s
// before it stores any r_s (the stores could alias the later loads as far as
// the compiler knows, which would serialise one memory round trip per line).
__device__ __forceinline__ float split_one(float r, float p, float pl, float fs)
{
    return (p > 1e-30f) ? r * (pl / p) : r * fs;
}

template <bool DET, bool XT = false>
__global__ void __launch_bounds__(256) k_split(const EprConsts C, const SplatArgs A)
{
    const int b = blockIdx.y;
    epr_grid_wait();
    if (A.check_done && A.st[b].done) return;
    epr_grid_release();
    const int ns = C.ns;
    const size_t npix = (size_t)C.nx * C.ny, pb = (size_t)b * npix;
    if constexpr (!DET) {   // nx % 4 == 0: four pixels of one row per thread
        const size_t n4 = npix / 4;
        for (size_t q4 = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q4 < n4;
             q4 += (size_t)gridDim.x * blockDim.x) {
            const size_t q = 4 * q4;
            const float4 d = __ldg(reinterpret_cast<const float4*>(A.D + pb + q));
            const float4 p = *reinterpret_cast<const float4*>(A.P + pb + q);
            const float4 r = make_float4(d.x - p.x, d.y - p.y, d.z - p.z, d.w - p.w);
            const int x = (int)(q % (size_t)C.nx);
            float4 pl[EPR_MAX_LINES];
#pragma unroll
            for (int s = 0; s < EPR_MAX_LINES; ++s)
                if (s < ns && ns > 1)
                    pl[s] = *reinterpret_cast<const float4*>(A.Ps + (pb * ns) + (size_t)s * npix + q);
#pragma unroll
            for (int s = 0; s < EPR_MAX_LINES; ++s) {
                if (!(s < ns && ns > 1)) continue;
                float4 o;
                if constexpr (XT) {
                    o = make_float4(split_one(r.x, p.x, pl[s].x, xt_get(C, EPR_XT_F, s, x)),
                                    split_one(r.y, p.y, pl[s].y, xt_get(C, EPR_XT_F, s, x + 1)),
                                    split_one(r.z, p.z, pl[s].z, xt_get(C, EPR_XT_F, s, x + 2)),
                                    split_one(r.w, p.w, pl[s].w, xt_get(C, EPR_XT_F, s, x + 3)));
                } else {
                    const float fs = C.f[s];
                    o = make_float4(split_one(r.x, p.x, pl[s].x, fs), split_one(r.y, p.y, pl[s].y, fs),
                                    split_one(r.z, p.z, pl[s].z, fs), split_one(r.w, p.w, pl[s].w, fs));
                }
                *reinterpret_cast<float4*>(A.Ps + (pb * ns) + (size_t)s * npix + q) = o;
            }
            *reinterpret_cast<float4*>(A.P + pb + q) = r;
        }
        return;
    }
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < npix;
         q += (size_t)gridDim.x * blockDim.x) {
        const float d = __ldg(&A.D[pb + q]);
        const float p = DET ? (float)A.Pq[pb + q] * EPR_FX_INV : A.P[pb + q];
        const float r = d - p;
        for (int s = 0; ns > 1 && s < ns; ++s) {   // one line: r itself
            const size_t o = (pb * ns) + (size_t)s * npix + q;
            const float pl = DET ? (float)A.Psq[o] * EPR_FX_INV : A.Ps[o];
            const float fs = XT ? xt_get(C, EPR_XT_F, s, (int)(q % (size_t)C.nx)) : line_const(C.f, s);
            A.Ps[o] = split_one(r, p, pl, fs);
        }
        A.P[pb + q] = r;
    }
}

// Oversampled grid (os > 1): the detector image of the model is the mean of
// each os x os block of the fine P; the residual D - mean is formed per
// detector pixel and replicated to the fine pixels of its block, where it is
// split over the lines with the fine weights P_s / P.  One thread per
// detector pixel; P <- replicated residual, P_s <- split residuals.
template <bool DET>
__global__ void __launch_bounds__(256) k_split_os(const EprConsts C, const SplatArgs A)
{
    const int b = blockIdx.y;
    epr_grid_wait();
    if (A.check_done && A.st[b].done) return;
    epr_grid_release();
    const int ns = C.ns, os = C.os, nx = C.nx;
    const int nxd = C.nx / os, nyd = C.ny / os;
    const size_t npix = (size_t)C.nx * C.ny, pb = (size_t)b * npix;
    const size_t npd = (size_t)nxd * nyd;
    const float inv_o2 = 1.f / (float)(os * os);
    for (size_t qd = (size_t)blockIdx.x * blockDim.x + threadIdx.x; qd < npd;
         qd += (size_t)gridDim.x * blockDim.x) {
        const int yd = (int)(qd / nxd), xd = (int)(qd - (size_t)yd * nxd);
        const size_t f0 = pb + (size_t)yd * os * nx + (size_t)xd * os;   // block corner
        float mean;
        if constexpr (DET) {
            unsigned long long q = 0ull;
            for (int a = 0; a < os; ++a)
                for (int c = 0; c < os; ++c) q += A.Pq[f0 + (size_t)a * nx + c];
            mean = (float)q * EPR_FX_INV * inv_o2;
        } else {
            float sum = 0.f;
            for (int a = 0; a < os; ++a)
                for (int c = 0; c < os; ++c) sum += A.P[f0 + (size_t)a * nx + c];
            mean = sum * inv_o2;
        }
        const float r = __ldg(&A.D[(size_t)b * npd + qd]) - mean;
        for (int a = 0; a < os; ++a)
            for (int c = 0; c < os; ++c) {
                const size_t i = f0 + (size_t)a * nx + c;
                if (ns > 1) {
                    const float p = DET ? (float)A.Pq[i] * EPR_FX_INV : A.P[i];
                    for (int s = 0; s < ns; ++s) {
                        const size_t o = pb * ns + (size_t)s * npix + (i - pb);
                        const float pl = DET ? (float)A.Psq[o] * EPR_FX_INV : A.Ps[o];
                        A.Ps[o] = (p > 1e-30f) ? r * (pl / p) : r * line_const(C.f, s);
                    }
                }
                A.P[i] = r;
            }
    }
}

// Detector image of the forward model on an oversampled grid: the mean of
// each os x os block of P (out) and of each P_s (outs, may be NULL).
template <bool DET>
__global__ void __launch_bounds__(256) k_bin_os(const EprConsts C, const SplatArgs A, float* out,
                                                float* outs)
{
    const int b = blockIdx.y;
    const int ns = C.ns, os = C.os, nx = C.nx;
    const int nxd = C.nx / os, nyd = C.ny / os;
    const size_t npix = (size_t)C.nx * C.ny, pb = (size_t)b * npix;
    const size_t npd = (size_t)nxd * nyd;
    const float inv_o2 = 1.f / (float)(os * os);
    for (size_t qd = (size_t)blockIdx.x * blockDim.x + threadIdx.x; qd < npd;
         qd += (size_t)gridDim.x * blockDim.x) {
        const int yd = (int)(qd / nxd), xd = (int)(qd - (size_t)yd * nxd);
        const size_t f0 = (size_t)yd * os * nx + (size_t)xd * os;
        for (int s = -1; s < (outs ? ns : 0); ++s) {   // s = -1: P
            const bool tot = s < 0;
            const size_t base = tot ? pb : (pb * ns + (size_t)s * npix);
            if (!tot && ns == 1) {   // one line: P_s is P
                outs[(size_t)b * npd + qd] = out[(size_t)b * npd + qd];
                continue;
            }
            float m;
            if constexpr (DET) {
                const unsigned long long* q = tot ? A.Pq : A.Psq;
                unsigned long long sum = 0ull;
                for (int a = 0; a < os; ++a)
                    for (int c = 0; c < os; ++c) sum += q[base + f0 + (size_t)a * nx + c];
                m = (float)sum * EPR_FX_INV * inv_o2;
            } else {
                const float* q = tot ? A.P : A.Ps;
                float sum = 0.f;
                for (int a = 0; a < os; ++a)
                    for (int c = 0; c < os; ++c) sum += q[base + f0 + (size_t)a * nx + c];
                m = sum * inv_o2;
            }
            if (tot) out[(size_t)b * npd + qd] = m;
            else outs[((size_t)b * ns + s) * npd + qd] = m;
        }
    }
}

template <int NS, bool DET, bool RESID, int TH, int TW, int RC = 0, bool XT = false, int OCC = 0>
cudaError_t launch_t(const EprConsts& C, const SplatArgs& A, dim3 grid, size_t smem, int batch,
                     cudaStream_t stream)
{
    const bool pdl = C.pdl != 0;
    const cudaError_t e = epr_launch_kernel(pdl, k_splat<NS, DET, RESID, TH, TW, RC, XT, OCC>, grid,
                                            dim3(splat_threads(NS)), smem, stream, C, A);
    if (e != cudaSuccess) return e;
    return epr_launch_kernel(pdl, k_splat_overflow<DET, RESID, XT>, dim3(128, batch), dim3(128), 0,
                             stream, C, A);
}

// Tiles whose one-line residual kernel has a six-blocks-per-SM variant.
template <int TH, int TW>
constexpr bool has_occ6() { return TH * TW < 64 * 64; }

template <int TH, int TW>
cudaError_t launch_shape(const EprConsts& C, const SplatArgs& A, int resid, bool occ6, dim3 grid,
                         size_t smem, int batch, cudaStream_t stream)
{
    const bool mono = C.ns == 1;
    if (C.xt)   // x-dependent spectrum: the generic kernels with per-column constants
        return C.det ? launch_t<0, true, false, TH, TW, 0, true>(C, A, grid, smem, batch, stream)
                     : launch_t<0, false, false, TH, TW, 0, true>(C, A, grid, smem, batch, stream);
    if (C.det)
        return mono ? launch_t<1, true, false, TH, TW>(C, A, grid, smem, batch, stream)
                    : launch_t<0, true, false, TH, TW>(C, A, grid, smem, batch, stream);
    if constexpr (has_occ6<TH, TW>()) {
        if (resid && mono && occ6 && C.smax == 3)
            return launch_t<1, false, true, TH, TW, 3, false, 6>(C, A, grid, smem, batch, stream);
        if (resid && mono && occ6 && C.smax == 4)
            return launch_t<1, false, true, TH, TW, 4, false, 6>(C, A, grid, smem, batch, stream);
    }
    if (resid && mono) {
        switch (C.smax) {
        case 3: return launch_t<1, false, true, TH, TW, 3>(C, A, grid, smem, batch, stream);
        case 4: return launch_t<1, false, true, TH, TW, 4>(C, A, grid, smem, batch, stream);
        case 6: return launch_t<1, false, true, TH, TW, 6>(C, A, grid, smem, batch, stream);
        default: return launch_t<1, false, true, TH, TW>(C, A, grid, smem, batch, stream);
        }
    }
    if (mono) return launch_t<1, false, false, TH, TW>(C, A, grid, smem, batch, stream);
    if (C.ns == 8)   // the common polychromatic counts with an unrolled line loop
        return C.smax == 4 ? launch_t<8, false, false, TH, TW, 4>(C, A, grid, smem, batch, stream)
                           : launch_t<8, false, false, TH, TW>(C, A, grid, smem, batch, stream);
    if (C.ns == 4)
        return C.smax == 4 ? launch_t<4, false, false, TH, TW, 4>(C, A, grid, smem, batch, stream)
                           : launch_t<4, false, false, TH, TW>(C, A, grid, smem, batch, stream);
    switch (C.smax) {
    case 3: return launch_t<0, false, false, TH, TW, 3>(C, A, grid, smem, batch, stream);
    case 4: return launch_t<0, false, false, TH, TW, 4>(C, A, grid, smem, batch, stream);
    case 6: return launch_t<0, false, false, TH, TW, 6>(C, A, grid, smem, batch, stream);
    default: return launch_t<0, false, false, TH, TW>(C, A, grid, smem, batch, stream);
    }
}

template <int TH, int TW>
cudaError_t init_shape()
{
    cudaError_t e = epr_allow_max_smem(k_splat<1, true, false, TH, TW>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_splat<0, true, false, TH, TW>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_splat<1, false, true, TH, TW>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_splat<1, false, true, TH, TW, 3>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_splat<1, false, true, TH, TW, 4>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_splat<1, false, true, TH, TW, 6>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_splat<1, false, false, TH, TW>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_splat<0, false, false, TH, TW>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_splat<0, false, false, TH, TW, 3>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_splat<0, false, false, TH, TW, 4>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_splat<0, false, false, TH, TW, 6>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_splat<8, false, false, TH, TW, 4>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_splat<8, false, false, TH, TW>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_splat<4, false, false, TH, TW, 4>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_splat<4, false, false, TH, TW>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_splat<0, true, false, TH, TW, 0, true>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_splat<0, false, false, TH, TW, 0, true>);
    if constexpr (has_occ6<TH, TW>()) {
        if (e == cudaSuccess) e = epr_allow_max_smem(k_splat<1, false, true, TH, TW, 3, false, 6>);
        if (e == cudaSuccess) e = epr_allow_max_smem(k_splat<1, false, true, TH, TW, 4, false, 6>);
    }
    return e;
}

}  // namespace

// Whether the six-blocks-per-SM residual splat exists for this tile and reach.
bool epr_splat_has_occ6(int TH, int TW, int reach) { return TH * TW < 64 * 64 && (reach == 3 || reach == 4); }

size_t epr_splat_smem(const EprConsts& C, int TH, int TW)
{
    const int R = C.smax + 1;
    const int HX = (R + 1 + 3) & ~3;
    const int SH = (TH + 2 * R + kQuad - 1) / kQuad * kQuad + 2;
    const size_t acc_bytes = (size_t)C.ns * (TH + 2) * (TW + 2) * (C.det ? 8 : 4);
    return ((acc_bytes + 15) & ~size_t(15)) + (size_t)SH * (TW + 2 * HX) * sizeof(float);
}

// Host launcher: the tile kernel, then the overflow kernel (2 launches).
// resid = 1 (mono float only): P receives D - P.  `parity` alternates the
// overflow counter slot between consecutive splats of a solve.
cudaError_t epr_launch_splat(const EprConsts& C, const EprWork& W, const float* T, const float* D,
                             int resid, int parity, int batch, int TH, int TW, int check_done,
                             cudaStream_t stream)
{
    SplatArgs A;
    A.T = T;
    A.D = D;
    A.P = W.P;
    A.Ps = W.Ps;
    A.Pq = W.Pq;
    A.Psq = W.Psq;
    A.ovf_idx = W.ovf_idx;
    A.ovf_mask = W.ovf_mask;
    A.ovf_tg = W.ovf_tg;
    A.st = W.st;
    A.err = W.err;
    A.parity = parity & 1;
    A.check_done = check_done;
    {   // 2^(32 - S) >= 2 (2 reach + 3)^2: the largest pixel sum fits in uint32
        const int win = 2 * (2 * C.smax + 3) * (2 * C.smax + 3);
        int bits = 0;
        while ((1 << bits) < win) ++bits;
        A.fxs = ldexpf(1.f, 32 - bits);
        A.fxs_inv = ldexpf(1.f, bits - 32);
    }
    const size_t smem = epr_splat_smem(C, TH, TW);
    dim3 grid((C.nx + TW - 1) / TW, (C.ny + TH - 1) / TH, batch);
    cudaError_t e;
    if (TH == 64 && TW == 64) e = launch_shape<64, 64>(C, A, resid, W.splat_occ6 != 0, grid, smem, batch, stream);
    else if (TH == 32 && TW == 64) e = launch_shape<32, 64>(C, A, resid, W.splat_occ6 != 0, grid, smem, batch, stream);
    else if (TH == 64 && TW == 32) e = launch_shape<64, 32>(C, A, resid, W.splat_occ6 != 0, grid, smem, batch, stream);
    else if (TH == 32 && TW == 32) e = launch_shape<32, 32>(C, A, resid, W.splat_occ6 != 0, grid, smem, batch, stream);
    else return cudaErrorInvalidValue;
    epr_count_launch(2);
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t epr_splat_init()
{
    cudaError_t e = init_shape<64, 64>();
    if (e == cudaSuccess) e = init_shape<32, 64>();
    if (e == cudaSuccess) e = init_shape<64, 32>();
    if (e == cudaSuccess) e = init_shape<32, 32>();
    return e;
}

// Residual split after the forward of a solve: fixed_point = 1 reads the
// integer sums of the fixed-point splat, 0 the float maps (float splat,
// local closure).
cudaError_t epr_launch_split(const EprConsts& C, const EprWork& W, const float* D, int batch,
                             int fixed_point, int check_done, cudaStream_t stream)
{
    SplatArgs A = {};
    A.D = D;
    A.P = W.P;
    A.Ps = W.Ps;
    A.Pq = W.Pq;
    A.Psq = W.Psq;
    A.st = W.st;
    A.check_done = check_done;
    const size_t npix = (size_t)C.nx * C.ny;
    size_t blocks = (npix + 255) / 256;
    if (blocks > 1216) blocks = 1216;   // 8 per SM on 152 SMs, grid-stride beyond
    const dim3 grid((unsigned)blocks, batch);
    cudaError_t e;
    if (C.xt)
        e = fixed_point ? epr_launch_kernel(C.pdl != 0, k_split<true, true>, grid, dim3(256), 0, stream, C, A)
                        : epr_launch_kernel(C.pdl != 0, k_split<false, true>, grid, dim3(256), 0, stream, C, A);
    else
        e = fixed_point ? epr_launch_kernel(C.pdl != 0, k_split<true>, grid, dim3(256), 0, stream, C, A)
                        : epr_launch_kernel(C.pdl != 0, k_split<false>, grid, dim3(256), 0, stream, C, A);
    epr_count_launch(1);
    return e != cudaSuccess ? e : cudaGetLastError();
}

// Oversampled solve: the split at detector resolution (k_split_os).
cudaError_t epr_launch_split_os(const EprConsts& C, const EprWork& W, const float* D, int batch,
                                int fixed_point, int check_done, cudaStream_t stream)
{
    SplatArgs A = {};
    A.D = D;
    A.P = W.P;
    A.Ps = W.Ps;
    A.Pq = W.Pq;
    A.Psq = W.Psq;
    A.st = W.st;
    A.check_done = check_done;
    const size_t npd = (size_t)(C.nx / C.os) * (C.ny / C.os);
    size_t blocks = (npd + 255) / 256;
    if (blocks > 1216) blocks = 1216;
    const dim3 grid((unsigned)blocks, batch), blk(256);
    const bool pdl = C.pdl != 0;
    const cudaError_t e =
        fixed_point ? epr_launch_kernel(pdl, k_split_os<true>, grid, blk, 0, stream, C, A)
                    : epr_launch_kernel(pdl, k_split_os<false>, grid, blk, 0, stream, C, A);
    epr_count_launch(1);
    return e != cudaSuccess ? e : cudaGetLastError();
}

// Oversampled forward: detector images of P and of each P_s (outs may be NULL).
cudaError_t epr_launch_bin_os(const EprConsts& C, const EprWork& W, int fixed_point, float* out,
                              float* outs, int batch, cudaStream_t stream)
{
    SplatArgs A = {};
    A.P = W.P;
    A.Ps = W.Ps;
    A.Pq = W.Pq;
    A.Psq = W.Psq;
    const size_t npd = (size_t)(C.nx / C.os) * (C.ny / C.os);
    size_t blocks = (npd + 255) / 256;
    if (blocks > 1216) blocks = 1216;
    const dim3 grid((unsigned)blocks, batch), blk(256);
    if (fixed_point) k_bin_os<true><<<grid, blk, 0, stream>>>(C, A, out, outs);
    else k_bin_os<false><<<grid, blk, 0, stream>>>(C, A, out, outs);
    epr_count_launch(1);
    return cudaGetLastError();
}

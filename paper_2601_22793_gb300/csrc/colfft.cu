// Column pass of the 2-D preconditioner: forward FFT along y, the
// FFT-diagonal Paganin-type filter H_s(q) = mu_s / (mu_s + L delta_s |q|^2)
// (arXiv 2601.22793, "Linear term and relation to Paganin"; the approximate
// inverse P_{1,s}^{-1} applied in "Iteration structure"), inverse FFT along y.
// The 1 / (nx ny) normalisation of the two inverse transforms is folded into
// the filter.
//
// One block transforms CW adjacent columns of the packed half spectrum of
// one (projection, line); the tile [ny][CW] lives in shared memory.  Column 0
// holds two real-input columns packed as one complex column (X[0] in the
// real part, the Nyquist X[nx/2] in the imaginary part); after the forward
// transform the two are separated with C[ky] and conj C[-ky], filtered with
// their own symbols and packed again:
//   C'[ky] = (H0 + HN)/2 C[ky] + (H0 - HN)/2 conj C[-ky].
#include <cudaTypedefs.h>

#include "epr_internal.cuh"
#include "fft.cuh"
#include "tma.cuh"

int epr_row_blocks(const EprConsts& C);

namespace {

using PC = eprfft::PadCol;  // shared layout of the column tile

struct ColArgs {
    float2* S;            // [B][nl][ny][nx/2]
    EprProjState* st;
    const float2* tw;     // exp(-2 pi i t / ny)
    unsigned int* err;    // device error word
    const double* part_c; // [B][max_blocks] forward row pass partials
    double* rho_hist;     // [B][hist_len]
    int CW, lgCW;
    int line0, nl;
    int check_done;
    int rho_it;           // >= 0: block 0 forms rho of this iteration
    int nblk, max_blocks, hist_len;
    int kind;             // symbol of the generic pass: 0 = H = 1 / (1 + a),
                          // 1, 2 = kscale a / (1 + a)^2 (the derivatives of
                          // H by mu and by L delta), a = (L delta / mu) |q|^2
    float kscale;         // 1 / mu (kind 1) or -1 / (L delta) (kind 2)
};

// Symbol of the generic column pass at a = (L delta / mu) |q|^2, times the
// 1 / (nx ny) of the two inverse transforms.  With H = mu / (mu + L delta
// |q|^2) = 1 / (1 + a): dH/dmu = (a / mu) / (1 + a)^2 and dH/d(L delta) =
// -(a / (L delta)) / (1 + a)^2.
__device__ __forceinline__ float col_symbol(const ColArgs& A, float inv_n, float a)
{
    if (A.kind == 0) return inv_n / (1.f + a);
    const float d = 1.f + a;
    return A.kscale * inv_n * a / (d * d);
}

// Block 0 of the column pass of a solve (line 0) turns the forward row
// pass's partials into rho; the grid dependency wait has made them visible.
__device__ __forceinline__ void col_finalize_rho(const ColArgs& A, int b, bool lead)
{
    if (A.rho_it >= 0 && lead)
        finalize_rho(&A.st[b], A.part_c + (size_t)b * A.max_blocks, A.nblk,
                     A.rho_hist ? A.rho_hist + (size_t)b * A.hist_len : nullptr, A.hist_len, A.rho_it);
}

// The Paganin filter H = inv_n / (1 + ha kx^2 + hb ky^2) of element e of a
// [NY][CW] tile whose first column is kx0 > 0, as the output map of the last
// forward FFT stage (a fast reciprocal: 2 ulp).
template <int NY, int CW, int LGCW>
struct ColPaganin {
    float ha, hb, inv_n;
    int kx0;
    __device__ __forceinline__ float2 operator()(float2 v, int e) const
    {
        const int y = e >> LGCW, c = e & (CW - 1);
        const float ky = (float)(y <= NY / 2 ? y : y - NY), kx = (float)(kx0 + c);
        const float H = __fdividef(inv_n, fmaf(ha * kx, kx, fmaf(hb * ky, ky, 1.f)));
        return make_float2(v.x * H, v.y * H);
    }
};

// The filter of the tile holding column kx = 0, in place in buf.  That column
// packs the DC and Nyquist columns of the real transform, so its output at y
// mixes the values at y and NY - y: a thread takes both of a mirrored pair.
// The other columns of the tile are filtered pointwise.  Ends with a barrier.
template <int NY, int CW, int LGCW, int T>
__device__ __forceinline__ void col_filter0(float2* buf, const EprConsts& C, int s, int tid)
{
    const float ha = line_const(C.ha, s), hb = line_const(C.hb, s), inv_n = C.inv_n;
    const float kn = (float)C.half;
    for (int y = tid; y <= NY / 2; y += T) {
        const int yn = y == 0 ? 0 : NY - y;   // 0 and NY / 2 are their own mirror
        const float ky = (float)y;
        const float qy = hb * ky * ky;
        const float H0 = inv_n / (1.f + qy);
        const float HN = inv_n / (1.f + ha * kn * kn + qy);
        const float hp = 0.5f * (H0 + HN), hm = 0.5f * (H0 - HN);
        const float2 a = buf[eprfft::PadCol::idx(y << LGCW)];
        const float2 b = buf[eprfft::PadCol::idx(yn << LGCW)];
        buf[eprfft::PadCol::idx(y << LGCW)] = make_float2(hp * a.x + hm * b.x, hp * a.y - hm * b.y);
        if (yn != y)
            buf[eprfft::PadCol::idx(yn << LGCW)] = make_float2(hp * b.x + hm * a.x, hp * b.y - hm * a.y);
    }
    const ColPaganin<NY, CW, LGCW> f{ha, hb, inv_n, 0};
    for (int e = tid; e < NY * CW; e += T) {
        if ((e & (CW - 1)) == 0) continue;
        const int i = eprfft::PadCol::idx(e);
        buf[i] = f(buf[i], e);
    }
    __syncthreads();
}

template <int EPT>
__global__ void __launch_bounds__(512, 2) k_col(const EprConsts C, const ColArgs A)
{
    extern __shared__ __align__(16) float2 buf[];
    const int b = blockIdx.z, sl = blockIdx.y;
    epr_grid_wait();
    if (A.check_done && A.st[b].done) return;
    epr_grid_release();
    col_finalize_rho(A, b, blockIdx.x == 0 && sl == 0);
    const int s = A.line0 + sl;
    const int ny = C.ny, half = C.half, CW = A.CW, lgCW = A.lgCW;
    const int T = blockDim.x, tid = threadIdx.x;
    const int kx0 = blockIdx.x * CW;
    float2* Sb = A.S + ((size_t)b * A.nl + sl) * (size_t)ny * half;

    for (int e = tid; e < ny * CW; e += T) {
        const int y = e >> lgCW, c = e & (CW - 1);
        buf[PC::idx(e)] = Sb[(size_t)y * half + kx0 + c];
    }
    __syncthreads();
    eprfft::fft<PC, -1, EPT>(buf, ny, lgCW, CW, 1, A.tw, T, tid);

    // filter (two phases: column 0 reads the mirrored frequency)
    const float ha = C.ha[s], hb = C.hb[s], inv_n = C.inv_n;
    float2 nv[EPT];
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
        const int e = tid + k * T;
        const int y = e >> lgCW, c = e & (CW - 1);
        const int kx = kx0 + c;
        const float ky = (float)(y <= ny / 2 ? y : y - ny);
        const float qy = hb * ky * ky;
        const float2 v = buf[PC::idx(e)];
        if (kx != 0) {
            const float H = col_symbol(A, inv_n, ha * (float)kx * (float)kx + qy);
            nv[k] = cscale(v, H);
        } else {
            const float kn = (float)half;
            const float H0 = col_symbol(A, inv_n, qy);
            const float HN = col_symbol(A, inv_n, ha * kn * kn + qy);
            const int yneg = (y == 0) ? 0 : ny - y;
            const float2 w = cconj(buf[PC::idx((yneg << lgCW) + c)]);
            const float hp = 0.5f * (H0 + HN), hm = 0.5f * (H0 - HN);
            nv[k] = make_float2(hp * v.x + hm * w.x, hp * v.y + hm * w.y);
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < EPT; ++k) buf[PC::idx(tid + k * T)] = nv[k];
    __syncthreads();
    eprfft::fft<PC, +1, EPT>(buf, ny, lgCW, CW, 1, A.tw, T, tid);
    for (int e = tid; e < ny * CW; e += T) {
        const int y = e >> lgCW, c = e & (CW - 1);
        Sb[(size_t)y * half + kx0 + c] = buf[PC::idx(e)];
    }
}

// Compile-time column length NY and width CW, on the compile-time FFT engine.
template <int NY, int CW, int EPT>
__global__ void __launch_bounds__(NY * CW / EPT, (65536 / 64) / (NY * CW / EPT))
k_col_ct(const EprConsts C, const ColArgs A)
{
    constexpr int T = NY * CW / EPT;
    constexpr int LGCW = CW == 1 ? 0 : CW == 2 ? 1 : CW == 4 ? 2 : CW == 8 ? 3 : 4;
    extern __shared__ __align__(16) float2 buf[];
    const int b = blockIdx.z, sl = blockIdx.y;
    epr_grid_wait();
    if (A.check_done && A.st[b].done) return;
    col_finalize_rho(A, b, blockIdx.x == 0 && sl == 0);
    const int s = A.line0 + sl;
    const int half = C.half, tid = threadIdx.x;
    const int kx0 = blockIdx.x * CW;
    float2* Sb = A.S + ((size_t)b * A.nl + sl) * (size_t)NY * half;
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
        const int e = tid + k * T;
        const int y = e >> LGCW, c = e & (CW - 1);
        buf[PC::idx(e)] = Sb[(size_t)y * half + kx0 + c];
    }
    __syncthreads();
    if (kx0 != 0) {   // the filter as the output map of the forward transform
        const ColPaganin<NY, CW, LGCW> f{line_const(C.ha, s), line_const(C.hb, s), C.inv_n, kx0};
        eprfft::fft_ct<PC, -1, NY, EPT, LGCW, CW, 1, 0>(buf, A.tw, tid, f);
    } else {
        eprfft::fft_ct<PC, -1, NY, EPT, LGCW, CW, 1>(buf, A.tw, tid);
        col_filter0<NY, CW, LGCW, T>(buf, C, s, tid);
    }
    eprfft::fft_ct<PC, +1, NY, EPT, LGCW, CW, 1>(buf, A.tw, tid);
    epr_grid_release();
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
        const int e = tid + k * T;
        const int y = e >> LGCW, c = e & (CW - 1);
        Sb[(size_t)y * half + kx0 + c] = buf[PC::idx(e)];
    }
}

// The same pass with the [NY][CW] tile moved by the tensor memory
// accelerator: BOXES bulk loads of [NY / BOXES][CW] into a dense tile at the
// start of the FFT buffer (no L1 traffic, one elected thread).  The first
// FFT stage reads every operand from the dense tile before its barrier and
// writes the padded layout over it; the last stage reads the padded layout
// and writes its results dense over it, which the bulk store reads.  So the
// block needs only the padded buffer.  The tile's row pitch is
// CW * 8 bytes, which keeps the strided 16-byte row segments of the column
// off the load/store unit.
constexpr unsigned int kTmaWaitPolls = 1u << 22;

// OCC > 0: that many blocks per SM (the radix-16 2048-row pass at five: 48
// registers, no spills), else the default bound.
template <int NY, int CW, int EPT, int MAXR = 8, int OCC = 0>
__global__ void __launch_bounds__(NY * CW / EPT,
                                  OCC > 0 ? OCC : NY * CW / EPT == 512 ? 3 : (65536 / 64) / (NY * CW / EPT))
k_col_tma(const EprConsts C, const ColArgs A, const __grid_constant__ CUtensorMap map)
{
    constexpr int T = NY * CW / EPT;
    constexpr int LGCW = CW == 2 ? 1 : CW == 4 ? 2 : 3;
    constexpr int BOXY = NY < 256 ? NY : 256;
    constexpr int BOXES = NY / BOXY;
    constexpr unsigned int BYTES = NY * CW * sizeof(float2);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ alignas(8) uint64_t bar;
    // the 128-byte aligned FFT buffer; the dense tile occupies its start
    const size_t base = ((size_t)__cvta_generic_to_shared(smem_raw) + 127) & ~size_t(127);
    float2* buf = reinterpret_cast<float2*>(smem_raw + (base - (size_t)__cvta_generic_to_shared(smem_raw)));
    const int b = blockIdx.z, sl = blockIdx.y, tid = threadIdx.x;
    const int kx0 = blockIdx.x * CW;
    if (tid == 0) {
        epr_tma::mbar_init(&bar, 1);
        epr_tma::fence_async_shared();
    }
    __syncthreads();
    epr_grid_wait();
    if (A.check_done && A.st[b].done) return;
    const int row0 = (b * A.nl + sl) * NY;
    if (tid == 0) {
        epr_tma::fence_async_global();
        epr_tma::mbar_arrive_expect_tx(&bar, BYTES);
#pragma unroll
        for (int i = 0; i < BOXES; ++i)
            epr_tma::load_2d(buf + i * BOXY * CW, &map, 2 * kx0, row0 + i * BOXY, &bar);
    }
    col_finalize_rho(A, b, blockIdx.x == 0 && sl == 0);   // while the tile is in flight
    if (!epr_tma::mbar_wait(&bar, 0, kTmaWaitPolls)) {
        // the copy did not arrive: report, and wait once more (bounded) so
        // that no copy lands after the block has left
        if (tid == 0) atomicOr(A.err, EPR_DEVERR_TIMEOUT);
        epr_tma::mbar_wait(&bar, 0, kTmaWaitPolls);
        return;
    }
    const int s = A.line0 + sl;
    constexpr int NST = eprfft::ct_n_stages(NY, MAXR);
    // the inverse runs the reversed stage plan, whose first stage takes the
    // last forward stage's results as they are
    if (kx0 != 0) {   // last forward stage, filter, first inverse stage in registers
        const ColPaganin<NY, CW, LGCW> f{line_const(C.ha, s), line_const(C.hb, s), C.inv_n, kx0};
        eprfft::fft_ct_from_stages<PC, -1, NY, EPT, LGCW, CW, 1, NST - 1, MAXR>(buf, buf, A.tw, tid);
        eprfft::stage_turn<PC, -1, +1, EPT, NY, LGCW, CW, 1, MAXR>(buf, A.tw, tid, f);
        eprfft::fft_ct_rev_stages<PC, +1, NY, EPT, LGCW, CW, 1, 1, NST - 1, MAXR>(buf, A.tw, tid);
    } else {   // the packed DC / Nyquist column filters mirrored pairs in place
        eprfft::fft_ct_from<PC, -1, NY, EPT, LGCW, CW, 1, MAXR>(buf, buf, A.tw, tid);
        col_filter0<NY, CW, LGCW, T>(buf, C, s, tid);
        eprfft::fft_ct_rev_stages<PC, +1, NY, EPT, LGCW, CW, 1, 0, NST - 1, MAXR>(buf, A.tw, tid);
    }
    epr_grid_release();
    // the last stage writes the dense tile the bulk store reads, in place:
    // every operand is read before the stage's barrier
    eprfft::fft_ct_rev_last<eprfft::Dense, true, false, PC, +1, NY, EPT, LGCW, CW, 1, MAXR>(buf, A.tw, tid);
    epr_tma::fence_async_shared();
    __syncthreads();
    if (tid == 0) {
#pragma unroll
        for (int i = 0; i < BOXES; ++i)
            epr_tma::store_2d(&map, 2 * kx0, row0 + i * BOXY, buf + i * BOXY * CW);
        epr_tma::bulk_commit();
        epr_tma::bulk_wait_read_all();   // the tile must outlive the copy's reads
    }
}

}  // namespace

struct EprColLaunch {
    int CW, lgCW, EPT, threads;
    size_t smem;
};

EprColLaunch epr_col_config(const EprConsts& C, int cw_hint)
{
    EprColLaunch L;
    int cw = cw_hint > 0 ? cw_hint : 4;
    while (cw > 1 && C.half % cw != 0) cw >>= 1;
    // keep the block at 512 threads or fewer, 8 elements per thread if possible
    int ept = 8;
    // 8192-point columns (oversampled internal grids): one column, 1024 threads
    const int tmax = C.ny >= 8192 ? 1024 : 512;
    while (C.ny * cw / ept > tmax && cw > 1) cw >>= 1;
    while (C.ny * cw / ept > tmax && ept < 16) ept *= 2;
    L.CW = cw;
    L.lgCW = 0;
    while ((1 << L.lgCW) < cw) ++L.lgCW;
    L.EPT = ept;
    L.threads = C.ny * cw / ept;
    L.smem = (size_t)PC::len(C.ny * cw) * sizeof(float2);
    return L;
}

// The column passes that move their tile by bulk tensor copies.
// Column tile width of the bulk-copy pass: the plain pass's, except for
// 4096- and 8192-row columns (oversampled internal grids), whose bulk-copy
// tile is two columns wide (64 KB and 512 threads, or 128 KB and 1024
// threads, radix-16 stages) where the plain pass takes one.
static int col_tma_cw(const EprConsts& C, const EprColLaunch& L)
{
    return (C.ny == 4096 || C.ny == 8192) ? 2 : L.CW;
}

static bool col_tma_case(const EprConsts& C, const EprColLaunch& L)
{
    if (C.ny == 4096 || C.ny == 8192) return L.EPT == 8 && C.half % 2 == 0;
    if (L.EPT != 8) return false;
    return (L.CW == 4 && (C.ny == 256 || C.ny == 512 || C.ny == 1024)) ||
           (L.CW == 2 && (C.ny == 1536 || C.ny == 2048));
}

// elements per thread of the bulk-copy pass: 16 for 2048-point columns (256
// threads and 37 KB per block, four blocks per SM, so the 512 blocks of a
// 2048^2 projection are resident at once), 8 otherwise
static int col_tma_ept(const EprConsts& C) { return (C.ny == 2048 || C.ny >= 4096) ? 16 : 8; }

static size_t col_tma_smem(const EprConsts& C, const EprColLaunch& L)
{
    return 128 + (size_t)PC::len(C.ny * col_tma_cw(C, L)) * sizeof(float2);
}

// Tensor map of S seen as `rows` rows of nx floats, with [ny or 256][2 CW]
// boxes, for the bulk-copy column pass.  Returns false (and leaves the plain
// pass in use) when the size has no such pass or the CUDA driver API entry
// point cuTensorMapEncodeTiled is not available.
bool epr_col_make_map(const EprConsts& C, const float2* S, long long rows, CUtensorMap* out)
{
    const EprColLaunch L = epr_col_config(C, 0);
    if (!col_tma_case(C, L) || !S || rows <= 0 || rows > (1ll << 31)) return false;
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return false;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const cuuint64_t dims[2] = {(cuuint64_t)C.nx, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)C.nx * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)(2 * col_tma_cw(C, L)), (cuuint32_t)(C.ny < 256 ? C.ny : 256)};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = encode(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float2*>(S), dims,
                              strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// rho_it >= 0 (a solve): block 0 also forms rho of iteration rho_it from the
// forward row pass's partials.
cudaError_t epr_launch_col(const EprConsts& C, const EprWork& W, int line0, int nl, int batch,
                           int check_done, int cw_hint, int rho_it, cudaStream_t stream)
{
    const EprColLaunch L = epr_col_config(C, cw_hint);
    ColArgs A;
    A.S = W.S;
    A.st = W.st;
    A.tw = W.tw_y;
    A.err = W.err;
    A.part_c = W.part_c;
    A.rho_hist = W.rho_hist;
    A.rho_it = rho_it;
    A.nblk = rho_it >= 0 ? epr_row_blocks(C) : 0;
    A.max_blocks = W.max_blocks;
    A.hist_len = W.hist_len;
    A.CW = L.CW;
    A.lgCW = L.lgCW;
    A.line0 = line0;
    A.nl = nl;
    A.check_done = check_done;
    A.kind = 0;
    A.kscale = 0.f;
    const dim3 grid(C.half / L.CW, nl, batch);
    const bool pdl = C.pdl != 0;
    cudaError_t e = cudaSuccess;
    bool done = false;
    if (W.col_map && cw_hint == 0 && col_tma_case(C, L)) {
        const CUtensorMap& map = *static_cast<const CUtensorMap*>(W.col_map);
        const size_t smem = col_tma_smem(C, L);
        const int ept = col_tma_ept(C);
#define EPR_COL_TMA_CASE(NYV, CWV, EPTV)                                                       \
        if (!done && C.ny == NYV && L.CW == CWV && ept == EPTV) {                             \
            e = epr_launch_kernel(pdl, k_col_tma<NYV, CWV, EPTV>, grid, dim3(NYV * CWV / EPTV), \
                                  smem, stream, C, A, map);                                   \
            done = true;                                                                      \
        }
        EPR_COL_TMA_CASE(256, 4, 8)
        EPR_COL_TMA_CASE(512, 4, 8)
        EPR_COL_TMA_CASE(1024, 4, 8)
        EPR_COL_TMA_CASE(1536, 2, 8)
        if (!done && C.ny == 2048 && L.CW == 2 && ept == 16 && W.col_radix16) {
            e = W.col_occ5 ? epr_launch_kernel(pdl, k_col_tma<2048, 2, 16, 16, 5>, grid,
                                               dim3(2048 * 2 / 16), smem, stream, C, A, map)
                           : epr_launch_kernel(pdl, k_col_tma<2048, 2, 16, 16>, grid,
                                               dim3(2048 * 2 / 16), smem, stream, C, A, map);
            done = true;
        }
        if (!done && C.ny == 8192) {   // 2 columns per block, radix-16 stages 16, 16, 16, 2
            A.CW = 2;
            A.lgCW = 1;
            e = epr_launch_kernel(pdl, k_col_tma<8192, 2, 16, 16>, dim3(C.half / 2, nl, batch),
                                  dim3(8192 * 2 / 16), smem, stream, C, A, map);
            done = true;
        }
        if (!done && C.ny == 4096) {   // 2 columns per block, radix 16 (16, 16, 16), 2 blocks per SM
            A.CW = 2;
            A.lgCW = 1;
            e = epr_launch_kernel(pdl, k_col_tma<4096, 2, 16, 16, 2>, dim3(C.half / 2, nl, batch),
                                  dim3(4096 * 2 / 16), smem, stream, C, A, map);
            done = true;
        }
        EPR_COL_TMA_CASE(2048, 2, 16)
#undef EPR_COL_TMA_CASE
    }
#define EPR_COL_CASE(NYV, CWV, EPTV)                                                           \
    if (!done && C.ny == NYV && L.CW == CWV && L.EPT == EPTV) {                               \
        e = epr_launch_kernel(pdl, k_col_ct<NYV, CWV, EPTV>, grid, dim3(NYV * CWV / EPTV),    \
                              L.smem, stream, C, A);                                          \
        done = true;                                                                          \
    }
    EPR_COL_CASE(256, 4, 8)
    EPR_COL_CASE(512, 4, 8)
    EPR_COL_CASE(1024, 4, 8)
    EPR_COL_CASE(1536, 2, 8)
    EPR_COL_CASE(2048, 2, 8)
    EPR_COL_CASE(2048, 1, 8)
    EPR_COL_CASE(3072, 1, 8)
    EPR_COL_CASE(4096, 1, 8)
    EPR_COL_CASE(8192, 1, 8)
#undef EPR_COL_CASE
    if (!done) {
        if (L.EPT == 8)
            e = epr_launch_kernel(pdl, k_col<8>, grid, dim3(L.threads), L.smem, stream, C, A);
        else
            e = epr_launch_kernel(pdl, k_col<16>, grid, dim3(L.threads), L.smem, stream, C, A);
    }
    epr_count_launch(1);
    return e != cudaSuccess ? e : cudaGetLastError();
}

// The generic column pass with symbol `kind` (col_symbol) for one line of a
// batch of spectra (line slot 0 of S, the constants of line `line`): the
// filter derivatives of the reverse pass through the solve.
cudaError_t epr_launch_col_kind(const EprConsts& C, const EprWork& W, int line, int batch,
                                int kind, float kscale, cudaStream_t stream)
{
    const EprColLaunch L = epr_col_config(C, 0);
    ColArgs A = {};
    A.S = W.S;
    A.st = W.st;
    A.tw = W.tw_y;
    A.err = W.err;
    A.rho_it = -1;
    A.CW = L.CW;
    A.lgCW = L.lgCW;
    A.line0 = line;
    A.nl = 1;
    A.check_done = 0;
    A.kind = kind;
    A.kscale = kscale;
    const dim3 grid(C.half / L.CW, 1, batch);
    cudaError_t e;
    if (L.EPT == 8)
        e = epr_launch_kernel(false, k_col<8>, grid, dim3(L.threads), L.smem, stream, C, A);
    else
        e = epr_launch_kernel(false, k_col<16>, grid, dim3(L.threads), L.smem, stream, C, A);
    epr_count_launch(1);
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t epr_col_init()
{
    cudaError_t e = epr_allow_max_smem(k_col<8>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_col<16>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_col_ct<256, 4, 8>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_col_ct<512, 4, 8>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_col_ct<1024, 4, 8>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_col_ct<2048, 2, 8>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_col_ct<2048, 1, 8>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_col_tma<256, 4, 8>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_col_tma<512, 4, 8>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_col_tma<1024, 4, 8>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_col_tma<1536, 2, 8>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_col_tma<2048, 2, 16>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_col_tma<2048, 2, 16, 16>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_col_tma<2048, 2, 16, 16, 5>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_col_tma<8192, 2, 16, 16>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_col_tma<4096, 2, 16, 16, 2>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_col_ct<1536, 2, 8>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_col_ct<3072, 1, 8>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_col_ct<4096, 1, 8>);
    if (e == cudaSuccess) e = epr_allow_max_smem(k_col_ct<8192, 1, 8>);
    return e;
}

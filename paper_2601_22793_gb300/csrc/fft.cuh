// Shared-memory mixed-radix FFT engine (radix 8, 4, 2 and 3).
//
// Transforms `nseq` independent complex sequences of length N held in shared
// memory; element j of sequence m lives at buf[j * sj + m * sm].  The
// schedule is the Stockham autosort form: stage with radix R and running
// stride Ns reads buf[j + r N/R] (r < R), applies the twiddle
// exp(DIR 2 pi i r (j mod Ns) / (Ns R)), takes the R-point DFT and writes
// buf[(j / Ns) Ns R + (j mod Ns) + r Ns]; the output is in natural order.
// Each stage first reads every operand into registers, synchronises, then
// writes, so one buffer serves as input and output.
//
// Radices: as many 8 as divide N's power of two, then one 4 or 2, and the
// factors of 3 last, which keeps (j mod Ns) a bit mask except in the radix-3
// stages, where Ns = N / 3^k and j < Ns makes it j itself for the last one.
//
// The block has T threads with N * nseq = EPT * T, nseq a power of two;
// butterfly b of a stage maps to sequence b & (nseq-1) and index b >> lgseq.
// Twiddles come from a table tw[t] = exp(-2 pi i t / N) (float, built in
// double on the host); DIR = +1 uses its conjugate.  No normalisation.
//
// Shared-memory addresses pass through a layout policy PAD (PAD::idx(i)),
// and callers size and index their buffers with the same policy.  A 64-bit
// shared access is served per half-warp, 16 complex values (128 bytes) per
// wavefront, so the policies keep 16 consecutive values in distinct banks
// and spread the strided Stockham stores:
//  * PadRow (one sequence laid out contiguously, the row passes): an XOR
//    swizzle of the low four bits by the 128-byte row index (and, every
//    four rows, its bit 3) makes the stride-8 and stride-64 stores of the
//    first two radix-8 stages conflict-free; no extra space.
//  * PadCol (CW interleaved columns, the column pass): two padding values
//    after every sixteen, i + 2 (i / 16).
#pragma once

#include "epr_internal.cuh"

namespace eprfft {

// Each policy also states a period P and the address step of adding a
// multiple c of P to an index: idx(i + c) = idx(i) + step(c) for every i.  A
// stage whose operand stride is a multiple of P computes one address and adds
// constants.
struct PadRow {
    __host__ __device__ static __forceinline__ int idx(int i)
    {
        return (i & ~15) | ((i & 15) ^ (((i >> 4) & 7) ^ (((i >> 6) & 1) << 3)));
    }
    __host__ __device__ static __forceinline__ int len(int n) { return (n + 15) & ~15; }
    static constexpr int kPeriod = 128;   // the swizzle reads bits 0..6 only
    __host__ __device__ static constexpr int step(int c) { return c; }
};

struct PadCol {
    __host__ __device__ static __forceinline__ int idx(int i) { return i + 2 * (i >> 4); }
    __host__ __device__ static __forceinline__ int len(int n) { return n + 2 * (n >> 4) + 2; }
    static constexpr int kPeriod = 16;
    __host__ __device__ static constexpr int step(int c) { return c + 2 * (c >> 4); }
};

// Plain dense layout (a tile written by a bulk copy).
struct Dense {
    __host__ __device__ static __forceinline__ int idx(int i) { return i; }
    __host__ __device__ static __forceinline__ int len(int n) { return n; }
    static constexpr int kPeriod = 1;
    __host__ __device__ static constexpr int step(int c) { return c; }
};

// R-point DFTs in registers, sign DIR (-1 forward, +1 inverse).
template <int DIR>
__device__ __forceinline__ void dft2(float2& a, float2& b)
{
    float2 t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

// multiply by DIR * i
template <int DIR>
__device__ __forceinline__ float2 mul_i(float2 a)
{
    return DIR < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

template <int DIR>
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3)
{
    float2 t0 = cadd(a0, a2), t1 = csub(a0, a2);
    float2 t2 = cadd(a1, a3), t3 = mul_i<DIR>(csub(a1, a3));
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    a1 = cadd(t1, t3);
    a3 = csub(t1, t3);
}

template <int DIR>
__device__ __forceinline__ void dft8(float2* v)
{
    const float h = 0.70710678118654752440f;
    // even / odd halves
    dft4<DIR>(v[0], v[2], v[4], v[6]);
    dft4<DIR>(v[1], v[3], v[5], v[7]);
    // twiddles exp(DIR 2 pi i k / 8) on the odd half, k = 1, 2, 3
    float2 o1 = v[3], o2 = v[5], o3 = v[7];
    // k = 1: (h, DIR h)
    o1 = make_float2(h * (o1.x - (float)DIR * o1.y), h * (o1.y + (float)DIR * o1.x));
    // k = 2: DIR i
    o2 = mul_i<DIR>(o2);
    // k = 3: (-h, DIR h)
    o3 = make_float2(-h * (o3.x + (float)DIR * o3.y), h * ((float)DIR * o3.x - o3.y));
    float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    float2 q0 = v[1];
    v[0] = cadd(e0, q0);
    v[4] = csub(e0, q0);
    v[1] = cadd(e1, o1);
    v[5] = csub(e1, o1);
    v[2] = cadd(e2, o2);
    v[6] = csub(e2, o2);
    v[3] = cadd(e3, o3);
    v[7] = csub(e3, o3);
}

template <int DIR>
__device__ __forceinline__ void dft3(float2& a0, float2& a1, float2& a2)
{
    const float s3 = 0.86602540378443864676f;  // sin(2 pi / 3)
    float2 t = cadd(a1, a2), d = csub(a1, a2);
    float2 m = make_float2(a0.x - 0.5f * t.x, a0.y - 0.5f * t.y);
    float2 rd = mul_i<DIR>(d);  // DIR i (a1 - a2)
    a0 = cadd(a0, t);
    a1 = make_float2(m.x + s3 * rd.x, m.y + s3 * rd.y);
    a2 = make_float2(m.x - s3 * rd.x, m.y - s3 * rd.y);
}

// 16-point DFT as 4 x 4: with n = 4 n1 + n2 and k = k1 + 4 k2,
// X[k1 + 4 k2] = sum_n2 W4^(n2 k2) W16^(n2 k1) sum_n1 W4^(n1 k1) x[4 n1 + n2]:
// four 4-point DFTs down the columns n2, twiddles W16^(n2 k1), four 4-point
// DFTs along the rows k1, and the 4 x 4 transpose of the result (register
// renaming).
template <int DIR>
__device__ __forceinline__ void dft16(float2* v)
{
    const float c1 = 0.92387953251128675613f;   // cos(pi / 8)
    const float s1 = 0.38268343236508977173f;   // sin(pi / 8)
    const float h = 0.70710678118654752440f;
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4<DIR>(v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]);
    // v[n2 + 4 k1] *= exp(DIR 2 pi i n2 k1 / 16)
    auto rot = [](float2 a, float c, float s) {   // a (c + i s)
        return make_float2(a.x * c - a.y * s, a.x * s + a.y * c);
    };
    const float d = (float)DIR;
    v[1 + 4] = rot(v[1 + 4], c1, d * s1);           // n2 k1 = 1
    v[1 + 8] = rot(v[1 + 8], h, d * h);             // 2
    v[1 + 12] = rot(v[1 + 12], s1, d * c1);         // 3
    v[2 + 4] = rot(v[2 + 4], h, d * h);             // 2
    v[2 + 8] = mul_i<DIR>(v[2 + 8]);                // 4
    v[2 + 12] = rot(v[2 + 12], -h, d * h);          // 6
    v[3 + 4] = rot(v[3 + 4], s1, d * c1);           // 3
    v[3 + 8] = rot(v[3 + 8], -h, d * h);            // 6
    v[3 + 12] = rot(v[3 + 12], -c1, -d * s1);       // 9
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft4<DIR>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
    // v[4 k1 + k2] holds X[k1 + 4 k2]
    float2 o[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) o[k1 + 4 * k2] = v[4 * k1 + k2];
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = o[k];
}

template <int R, int DIR>
__device__ __forceinline__ void dft(float2* v)
{
    if constexpr (R == 2) dft2<DIR>(v[0], v[1]);
    else if constexpr (R == 3) dft3<DIR>(v[0], v[1], v[2]);
    else if constexpr (R == 4) dft4<DIR>(v[0], v[1], v[2], v[3]);
    else if constexpr (R == 16) dft16<DIR>(v);
    else dft8<DIR>(v);
}

template <class PAD, int R, int DIR, int EPT>
__device__ __forceinline__ void stage(float2* buf, int N, int Ns, int lgNs, int lgseq, int sj,
                                      int sm, const float2* __restrict__ tw, int T, int tid)
{
    constexpr int PER = (EPT + R - 1) / R;
    const int NR = N / R;
    const int nb = NR << lgseq;
    const int twstep = N / (Ns * R);
    const int mmask = (1 << lgseq) - 1;
    float2 v[PER][R];
    int dst[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int b = tid + k * T;
        dst[k] = -1;
        if (b < nb) {
            const int m = b & mmask;
            const int j = b >> lgseq;
            const int jm = (lgNs >= 0) ? (j & (Ns - 1)) : (j % Ns);
            const int jd = (lgNs >= 0) ? (j >> lgNs) : (j / Ns);
            const int base = m * sm;
#pragma unroll
            for (int r = 0; r < R; ++r) v[k][r] = buf[PAD::idx((j + r * NR) * sj + base)];
#pragma unroll
            for (int r = 1; r < R; ++r) {
                float2 w = __ldg(&tw[r * jm * twstep]);
                if (DIR > 0) w.y = -w.y;
                v[k][r] = cmul(v[k][r], w);
            }
            dst[k] = (jd * Ns * R + jm) * sj + base;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        if (dst[k] >= 0) {
            dft<R, DIR>(v[k]);
#pragma unroll
            for (int r = 0; r < R; ++r) buf[PAD::idx(dst[k] + r * Ns * sj)] = v[k][r];
        }
    }
    __syncthreads();
}

// Full transform.  The caller synchronises before (data in buf) and may read
// buf right after return (the last stage ends with a barrier).
template <class PAD, int DIR, int EPT>
__device__ void fft(float2* buf, int N, int lgseq, int sj, int sm, const float2* __restrict__ tw,
                    int T, int tid)
{
    int rem2 = N, rem3 = 1;
    while (rem2 % 3 == 0) {
        rem2 /= 3;
        rem3 *= 3;
    }
    int Ns = 1, lgNs = 0;
    while (rem2 >= 8) {
        stage<PAD, 8, DIR, EPT>(buf, N, Ns, lgNs, lgseq, sj, sm, tw, T, tid);
        Ns *= 8; lgNs += 3; rem2 /= 8;
    }
    if (rem2 == 4) {
        stage<PAD, 4, DIR, EPT>(buf, N, Ns, lgNs, lgseq, sj, sm, tw, T, tid);
        Ns *= 4; lgNs += 2;
    } else if (rem2 == 2) {
        stage<PAD, 2, DIR, EPT>(buf, N, Ns, lgNs, lgseq, sj, sm, tw, T, tid);
        Ns *= 2; lgNs += 1;
    }
    while (rem3 > 1) {
        stage<PAD, 3, DIR, EPT>(buf, N, Ns, -1, lgseq, sj, sm, tw, T, tid);
        Ns *= 3; rem3 /= 3;
    }
}

}  // namespace eprfft

// ---------------------------------------------------------------------------
// Compile-time-sized variant of the same Stockham schedule.  N, the number of
// sequences (1 << LGSEQ), the strides SJ / SM and the elements per thread are
// template parameters, so every stage is unrolled, strides fold into address
// offsets, the first stage (Ns = 1) needs no twiddle, and a radix-R stage
// loads one twiddle w = exp(DIR 2 pi i jm / (Ns R)) and forms w^2 .. w^(R-1)
// by the Chebyshev three-term recurrence of cos and sin (a few ulp for
// R <= 8, well inside the transform's error).
// ---------------------------------------------------------------------------
namespace eprfft {

__host__ __device__ constexpr int ct_pow2_part(int n)
{
    while (n % 3 == 0) n /= 3;
    return n;
}
// Stage plans: as many stages of the largest radix maxr (8, or 16 for blocks
// with 16 elements per thread) as divide the power of two, then one stage of
// the remaining power of two, then the factors of 3.
__host__ __device__ constexpr int ct_n_stages(int n, int maxr = 8)
{
    int p = ct_pow2_part(n), c = 0;
    while (p >= maxr) { p /= maxr; ++c; }
    if (p > 1) ++c;
    int t = n / ct_pow2_part(n);
    while (t > 1) { t /= 3; ++c; }
    return c;
}
__host__ __device__ constexpr int ct_radix(int n, int s, int maxr = 8)
{
    int p = ct_pow2_part(n), k = 0;
    while (p >= maxr) {
        if (k == s) return maxr;
        p /= maxr;
        ++k;
    }
    if (p > 1) {
        if (k == s) return p;
        ++k;
    }
    return 3;
}
__host__ __device__ constexpr int ct_ns(int n, int s, int maxr = 8)
{
    int v = 1;
    for (int i = 0; i < s; ++i) v *= ct_radix(n, i, maxr);
    return v;
}

// The reversed plan: the same radices in the opposite order (a Stockham
// transform is valid for any order of the factors).
__host__ __device__ constexpr int ct_radix_rev(int n, int s, int maxr = 8)
{
    return ct_radix(n, ct_n_stages(n, maxr) - 1 - s, maxr);
}
__host__ __device__ constexpr int ct_ns_rev(int n, int s, int maxr = 8)
{
    int v = 1;
    for (int i = 0; i < s; ++i) v *= ct_radix_rev(n, i, maxr);
    return v;
}

// Output map of a stage: out = post(value, e) with e = j * SJ + m * SM the
// element's unpadded index; Identity leaves the value.
struct Identity {
    __device__ __forceinline__ float2 operator()(float2 v, int) const { return v; }
};

// Reads its operands from `in` (layout PADI) and writes post(result) to
// `buf` (layout PAD).  Every operand is read before the stage's first
// barrier, so in == buf works even when PADI != PAD.  STORE = false hands
// each result to post only (post(value, e) for its side effects, nothing is
// written); SYNC_END = false leaves out the closing barrier.
template <class PADI, class PAD, int R, int DIR, int EPT, int N, int NS, int LGSEQ, int SJ, int SM,
          class POST = Identity, bool STORE = true, bool SYNC_END = true>
__device__ __forceinline__ void stage_ct(const float2* in, float2* buf, const float2* __restrict__ tw,
                                         int tid, const POST& post = POST())
{
    constexpr int NSEQ = 1 << LGSEQ;
    constexpr int T = (N * NSEQ) / EPT;
    constexpr int PER = (EPT + R - 1) / R;
    constexpr int NR = N / R;
    constexpr int NB = NR * NSEQ;
    constexpr int TWSTEP = N / (NS * R);
    float2 v[PER][R];
    int dst[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int b = tid + k * T;
        dst[k] = -1;
        if (NB % T == 0 || b < NB) {
            const int m = b & (NSEQ - 1);
            const int j = b >> LGSEQ;
            const int jm = j % NS;
            const int jd = j / NS;
            const int base = m * SM;
            if constexpr ((NR * SJ) % PADI::kPeriod == 0) {
                const int i0 = PADI::idx(j * SJ + base);
#pragma unroll
                for (int r = 0; r < R; ++r) v[k][r] = in[i0 + PADI::step(r * NR * SJ)];
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) v[k][r] = in[PADI::idx((j + r * NR) * SJ + base)];
            }
            if constexpr (NS > 1) {
                // w^r = (cos r theta, sin r theta) by the three-term recurrence
                // x_{r+1} = 2 cos(theta) x_r - x_{r-1} (two multiply-adds per power);
                // a radix-16 stage runs it to w^7 only and takes w^8 = (w^4)^2 and
                // w^(8 + r) = w^8 w^r, which keeps every power within a few ulp
                float2 w = __ldg(&tw[jm * TWSTEP]);
                if (DIR > 0) w.y = -w.y;
                const float c2 = w.x + w.x;
                constexpr int RREC = R > 8 ? 8 : R;
                float2 wpow[RREC];
                wpow[0] = make_float2(1.f, 0.f);
                if constexpr (RREC > 1) wpow[1] = w;
#pragma unroll
                for (int r = 2; r < RREC; ++r)
                    wpow[r] = make_float2(fmaf(c2, wpow[r - 1].x, -wpow[r - 2].x),
                                          fmaf(c2, wpow[r - 1].y, -wpow[r - 2].y));
#pragma unroll
                for (int r = 1; r < RREC; ++r) v[k][r] = cmul(v[k][r], wpow[r]);
                if constexpr (R > 8) {
                    const float2 w8 = cmul(wpow[4], wpow[4]);
                    v[k][8] = cmul(v[k][8], w8);
#pragma unroll
                    for (int r = 9; r < R; ++r) v[k][r] = cmul(v[k][r], cmul(w8, wpow[r - 8]));
                }
            }
            dst[k] = (jd * NS * R + jm) * SJ + base;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        if (NB % T == 0 || dst[k] >= 0) {
            dft<R, DIR>(v[k]);
            if constexpr (!STORE) {
#pragma unroll
                for (int r = 0; r < R; ++r) post(v[k][r], dst[k] + r * NS * SJ);
            } else if constexpr ((NS * SJ) % PAD::kPeriod == 0) {
                const int o0 = PAD::idx(dst[k]);
#pragma unroll
                for (int r = 0; r < R; ++r)
                    buf[o0 + PAD::step(r * NS * SJ)] = post(v[k][r], dst[k] + r * NS * SJ);
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r)
                    buf[PAD::idx(dst[k] + r * NS * SJ)] = post(v[k][r], dst[k] + r * NS * SJ);
            }
        }
    }
    if constexpr (SYNC_END) __syncthreads();
}

// Stages S .. SEND - 1 of the transform, no output map.
template <class PAD, int DIR, int N, int EPT, int LGSEQ, int SJ, int SM, int S, int SEND, int MAXR = 8>
__device__ __forceinline__ void fft_ct_stages(float2* buf, const float2* __restrict__ tw, int tid)
{
    if constexpr (S < SEND) {
        stage_ct<PAD, PAD, ct_radix(N, S, MAXR), DIR, EPT, N, ct_ns(N, S, MAXR), LGSEQ, SJ, SM>(buf, buf,
                                                                                              tw, tid);
        fft_ct_stages<PAD, DIR, N, EPT, LGSEQ, SJ, SM, S + 1, SEND, MAXR>(buf, tw, tid);
    }
}

// The last stage alone, its input in layout PAD: the results go to buf in
// layout PADO (in place), or with STORE = false to post only.  Follows
// fft_ct_stages<..., 0, ct_n_stages(N, MAXR) - 1>.
template <class PADO, bool STORE, bool SYNC_END, class PAD, int DIR, int N, int EPT, int LGSEQ, int SJ,
          int SM, int MAXR = 8, class POST = Identity>
__device__ __forceinline__ void fft_ct_last(float2* buf, const float2* __restrict__ tw, int tid,
                                            const POST& post = POST())
{
    constexpr int S = ct_n_stages(N, MAXR) - 1;
    stage_ct<PAD, PADO, ct_radix(N, S, MAXR), DIR, EPT, N, ct_ns(N, S, MAXR), LGSEQ, SJ, SM, POST, STORE,
             SYNC_END>(buf, buf, tw, tid, post);
}

// Stages S .. SEND - 1 of the reversed plan, no output map.
template <class PAD, int DIR, int N, int EPT, int LGSEQ, int SJ, int SM, int S, int SEND, int MAXR = 8>
__device__ __forceinline__ void fft_ct_rev_stages(float2* buf, const float2* __restrict__ tw, int tid)
{
    if constexpr (S < SEND) {
        stage_ct<PAD, PAD, ct_radix_rev(N, S, MAXR), DIR, EPT, N, ct_ns_rev(N, S, MAXR), LGSEQ, SJ, SM>(
            buf, buf, tw, tid);
        fft_ct_rev_stages<PAD, DIR, N, EPT, LGSEQ, SJ, SM, S + 1, SEND, MAXR>(buf, tw, tid);
    }
}

// The last stage of the reversed plan (input layout PAD, output PADO in
// place, or post only with STORE = false).
template <class PADO, bool STORE, bool SYNC_END, class PAD, int DIR, int N, int EPT, int LGSEQ, int SJ,
          int SM, int MAXR = 8, class POST = Identity>
__device__ __forceinline__ void fft_ct_rev_last(float2* buf, const float2* __restrict__ tw, int tid,
                                                const POST& post = POST())
{
    constexpr int S = ct_n_stages(N, MAXR) - 1;
    stage_ct<PAD, PADO, ct_radix_rev(N, S, MAXR), DIR, EPT, N, ct_ns_rev(N, S, MAXR), LGSEQ, SJ, SM, POST,
             STORE, SYNC_END>(buf, buf, tw, tid, post);
}

// Stages 0 .. SEND - 1 of the transform with its input in a dense tile `in`
// (which may be buf itself), no output map.
template <class PAD, int DIR, int N, int EPT, int LGSEQ, int SJ, int SM, int SEND, int MAXR = 8>
__device__ __forceinline__ void fft_ct_from_stages(const float2* in, float2* buf,
                                                   const float2* __restrict__ tw, int tid)
{
    static_assert(SEND >= 1, "at least the first stage");
    stage_ct<Dense, PAD, ct_radix(N, 0, MAXR), DIR, EPT, N, 1, LGSEQ, SJ, SM>(in, buf, tw, tid);
    fft_ct_stages<PAD, DIR, N, EPT, LGSEQ, SJ, SM, 1, SEND, MAXR>(buf, tw, tid);
}

// The turn between a forward transform and the inverse of its pointwise
// image: the last stage of the forward plan (direction DIRF), the output map
// post, and the first stage of the reversed plan in direction DIRI, in
// registers.  The last forward stage (radix R, Ns = N / R) leaves butterfly b
// with elements j + r N / R of its sequence, which are the operands of the
// reversed plan's first stage (radix R, Ns = 1, no twiddles) for the same
// butterfly, in the same order.  Reads its operands before its first barrier
// (in place), writes the inverse stage's results to buf and synchronises.
template <class PAD, int DIRF, int DIRI, int EPT, int N, int LGSEQ, int SJ, int SM, int MAXR = 8,
          class POST = Identity>
__device__ __forceinline__ void stage_turn(float2* buf, const float2* __restrict__ tw, int tid,
                                           const POST& post = POST())
{
    constexpr int SL = ct_n_stages(N, MAXR) - 1;
    constexpr int R = ct_radix(N, SL, MAXR);
    constexpr int NS = ct_ns(N, SL, MAXR);
    static_assert(NS * R == N && ct_radix_rev(N, 0, MAXR) == R, "the turn's two stages");
    constexpr int NSEQ = 1 << LGSEQ;
    constexpr int T = (N * NSEQ) / EPT;
    constexpr int PER = (EPT + R - 1) / R;
    constexpr int NR = N / R;
    constexpr int NB = NR * NSEQ;
    constexpr int TWSTEP = N / (NS * R);
    float2 v[PER][R];
    int j_of[PER], m_of[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int b = tid + k * T;
        j_of[k] = -1;
        if (NB % T == 0 || b < NB) {
            const int m = b & (NSEQ - 1);
            const int j = b >> LGSEQ;   // j < NR = NS: j mod NS = j
            const int base = m * SM;
#pragma unroll
            for (int r = 0; r < R; ++r) v[k][r] = buf[PAD::idx((j + r * NR) * SJ + base)];
            if constexpr (NS > 1) {
                float2 w = __ldg(&tw[j * TWSTEP]);
                if (DIRF > 0) w.y = -w.y;
                const float c2 = w.x + w.x;
                constexpr int RREC = R > 8 ? 8 : R;
                float2 wpow[RREC];
                wpow[0] = make_float2(1.f, 0.f);
                if constexpr (RREC > 1) wpow[1] = w;
#pragma unroll
                for (int r = 2; r < RREC; ++r)
                    wpow[r] = make_float2(fmaf(c2, wpow[r - 1].x, -wpow[r - 2].x),
                                          fmaf(c2, wpow[r - 1].y, -wpow[r - 2].y));
#pragma unroll
                for (int r = 1; r < RREC; ++r) v[k][r] = cmul(v[k][r], wpow[r]);
                if constexpr (R > 8) {
                    const float2 w8 = cmul(wpow[4], wpow[4]);
                    v[k][8] = cmul(v[k][8], w8);
#pragma unroll
                    for (int r = 9; r < R; ++r) v[k][r] = cmul(v[k][r], cmul(w8, wpow[r - 8]));
                }
            }
            j_of[k] = j;
            m_of[k] = m;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        if (NB % T == 0 || j_of[k] >= 0) {
            const int j = j_of[k], base = m_of[k] * SM;
            dft<R, DIRF>(v[k]);
#pragma unroll
            for (int r = 0; r < R; ++r) v[k][r] = post(v[k][r], (j + r * NS) * SJ + base);
            dft<R, DIRI>(v[k]);
            // the reversed plan's first stage writes element j R + r
#pragma unroll
            for (int r = 0; r < R; ++r) buf[PAD::idx((j * R + r) * SJ + base)] = v[k][r];
        }
    }
    __syncthreads();
}

// The first stage with its operands in registers: for one sequence (nseq =
// 1) with EPT equal to the first radix R, thread tid's operands are elements
// tid + r N / R, r < R, and the stage has no twiddles.  Writes its results to
// buf (layout PAD) and synchronises; the caller has synchronised already if
// buf aliases data that other threads still read.  Stages 1.. follow as
// fft_ct<..., 1>.
template <class PAD, int DIR, int N, int EPT, int SJ, int MAXR = 8>
__device__ __forceinline__ void stage0_regs(float2 (&v)[EPT], float2* buf, int tid)
{
    constexpr int R = ct_radix(N, 0, MAXR);
    static_assert(R == EPT && ct_n_stages(N, MAXR) > 1, "operands of the first stage in registers");
    dft<R, DIR>(v);
    const int dst = tid * R * SJ;   // (j / Ns) Ns R + (j mod Ns) with Ns = 1, j = tid
#pragma unroll
    for (int r = 0; r < R; ++r) buf[PAD::idx(dst + r * SJ)] = v[r];
    __syncthreads();
}

// Stages S.. of the transform; the last one maps its outputs through post.
// MAXR = 16 takes radix-16 stages (blocks with at least 16 elements per thread).
template <class PAD, int DIR, int N, int EPT, int LGSEQ, int SJ, int SM, int S = 0, int MAXR = 8,
          class POST = Identity>
__device__ __forceinline__ void fft_ct(float2* buf, const float2* __restrict__ tw, int tid,
                                       const POST& post = POST())
{
    static_assert(MAXR <= EPT, "a stage's butterfly holds MAXR elements of one thread");
    if constexpr (S + 1 < ct_n_stages(N, MAXR)) {
        stage_ct<PAD, PAD, ct_radix(N, S, MAXR), DIR, EPT, N, ct_ns(N, S, MAXR), LGSEQ, SJ, SM>(buf, buf,
                                                                                              tw, tid);
        fft_ct<PAD, DIR, N, EPT, LGSEQ, SJ, SM, S + 1, MAXR>(buf, tw, tid, post);
    } else if constexpr (S + 1 == ct_n_stages(N, MAXR)) {
        stage_ct<PAD, PAD, ct_radix(N, S, MAXR), DIR, EPT, N, ct_ns(N, S, MAXR), LGSEQ, SJ, SM>(
            buf, buf, tw, tid, post);
    }
}

// The same transform with its input in a dense tile `in` (element j of
// sequence m at in[j * SJ + m * SM]), which may be buf itself; the result is
// in buf.
template <class PAD, int DIR, int N, int EPT, int LGSEQ, int SJ, int SM, int MAXR = 8,
          class POST = Identity>
__device__ __forceinline__ void fft_ct_from(const float2* in, float2* buf, const float2* __restrict__ tw,
                                            int tid, const POST& post = POST())
{
    if constexpr (ct_n_stages(N, MAXR) == 1) {
        stage_ct<Dense, PAD, ct_radix(N, 0, MAXR), DIR, EPT, N, 1, LGSEQ, SJ, SM>(in, buf, tw, tid, post);
    } else {
        stage_ct<Dense, PAD, ct_radix(N, 0, MAXR), DIR, EPT, N, 1, LGSEQ, SJ, SM>(in, buf, tw, tid);
        fft_ct<PAD, DIR, N, EPT, LGSEQ, SJ, SM, 1, MAXR>(buf, tw, tid, post);
    }
}

}  // namespace eprfft

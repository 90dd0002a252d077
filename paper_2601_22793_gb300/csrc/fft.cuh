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
// Shared-memory addresses pass through pidx(i) = i + i/8: one padding word
// after every eight complex values.  The first stages write with strides of
// 8 and 64 words, which otherwise fall into the same banks; with the padding
// those stores are spread over all banks.  Callers index the buffers through
// pidx too, and size them with padded_len().
#pragma once

#include "epr_internal.cuh"

namespace eprfft {

__host__ __device__ __forceinline__ int pidx(int i) { return i + (i >> 3); }
__host__ __device__ __forceinline__ int padded_len(int n) { return n + (n >> 3) + 1; }

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

template <int R, int DIR>
__device__ __forceinline__ void dft(float2* v)
{
    if constexpr (R == 2) dft2<DIR>(v[0], v[1]);
    else if constexpr (R == 3) dft3<DIR>(v[0], v[1], v[2]);
    else if constexpr (R == 4) dft4<DIR>(v[0], v[1], v[2], v[3]);
    else dft8<DIR>(v);
}

template <int R, int DIR, int EPT>
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
            for (int r = 0; r < R; ++r) v[k][r] = buf[pidx((j + r * NR) * sj + base)];
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
            for (int r = 0; r < R; ++r) buf[pidx(dst[k] + r * Ns * sj)] = v[k][r];
        }
    }
    __syncthreads();
}

// Full transform.  The caller synchronises before (data in buf) and may read
// buf right after return (the last stage ends with a barrier).
template <int DIR, int EPT>
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
        stage<8, DIR, EPT>(buf, N, Ns, lgNs, lgseq, sj, sm, tw, T, tid);
        Ns *= 8; lgNs += 3; rem2 /= 8;
    }
    if (rem2 == 4) {
        stage<4, DIR, EPT>(buf, N, Ns, lgNs, lgseq, sj, sm, tw, T, tid);
        Ns *= 4; lgNs += 2;
    } else if (rem2 == 2) {
        stage<2, DIR, EPT>(buf, N, Ns, lgNs, lgseq, sj, sm, tw, T, tid);
        Ns *= 2; lgNs += 1;
    }
    while (rem3 > 1) {
        stage<3, DIR, EPT>(buf, N, Ns, -1, lgseq, sj, sm, tw, T, tid);
        Ns *= 3; rem3 /= 3;
    }
}

}  // namespace eprfft

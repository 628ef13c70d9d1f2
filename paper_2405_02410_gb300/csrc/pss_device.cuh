// pss_device.cuh -- device building blocks of the sm_103a pseudo-spectral step:
// complex arithmetic, the counter-based Philox4x32-10 generator, in-register
// radix-2/4/8/16 DFTs and the shared-memory Stockham pass that strings them
// into length-N FFTs (the F and F^-1 of Eq. cubicexample, arXiv:2405.02410).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "pss_internal.h"

namespace pss {

// ---------------------------------------------------------------------------
// complex numbers (float2 / double2)
// ---------------------------------------------------------------------------

template <typename T> __device__ __forceinline__ cplx<T> mk(T x, T y) { cplx<T> r; r.x = x; r.y = y; return r; }
template <typename T> __device__ __forceinline__ cplx<T> cadd(cplx<T> a, cplx<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ cplx<T> csub(cplx<T> a, cplx<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ cplx<T> cmul(cplx<T> a, cplx<T> b) {
    return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T> __device__ __forceinline__ cplx<T> cconj(cplx<T> a) { return mk<T>(a.x, -a.y); }
template <typename T> __device__ __forceinline__ cplx<T> cscale(cplx<T> a, T s) { return mk<T>(a.x * s, a.y * s); }

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC'11): ten rounds of two 32x32 -> 64-bit products with a
// Weyl-sequence key schedule.
// ---------------------------------------------------------------------------
struct u32x4 { uint32_t x, y, z, w; };

__device__ __forceinline__ u32x4 philox4x32_10(u32x4 c, uint32_t k0, uint32_t k1) {
    constexpr uint32_t kMulA = 0xD2511F53u, kMulB = 0xCD9E8D57u;
    constexpr uint32_t kWeylA = 0x9E3779B9u, kWeylB = 0xBB67AE85u;
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t hiA = __umulhi(kMulA, c.x), loA = kMulA * c.x;
        const uint32_t hiB = __umulhi(kMulB, c.z), loB = kMulB * c.z;
        c = u32x4{hiB ^ c.y ^ k0, loB, hiA ^ c.w ^ k1, loA};
        k0 += kWeylA;
        k1 += kWeylB;
    }
    return c;
}

// u = ((x >> 8) + 0.5) / 2^24: exact in float and double, strictly inside (0, 1)
template <typename T> __device__ __forceinline__ T uniform24(uint32_t x) {
    return (T(x >> 8) + T(0.5)) * T(5.9604644775390625e-08);
}

// Box-Muller pair from two uniforms; sincospi(2 u1) gives cos/sin(2 pi u1) with
// an exact argument.
__device__ __forceinline__ void box_muller(float u0, float u1, float &n1, float &n2) {
    const float r = sqrtf(-2.0f * logf(u0));
    float s, c;
    sincospif(2.0f * u1, &s, &c);
    n1 = r * c;
    n2 = r * s;
}
__device__ __forceinline__ void box_muller(double u0, double u1, double &n1, double &n2) {
    const double r = sqrt(-2.0 * log(u0));
    double s, c;
    sincospi(2.0 * u1, &s, &c);
    n1 = r * c;
    n2 = r * s;
}

// ---------------------------------------------------------------------------
// 16th roots of unity: cos(2 pi k / 16) from the exact first-quadrant values.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr double cos16(int k) {
    k &= 15;
    // cos(pi/8), cos(pi/4), cos(3 pi/8)
    constexpr double c1 = 0.92387953251128675613, c2 = 0.70710678118654752440, c3 = 0.38268343236508977173;
    return k == 0 ? 1.0 : k == 1 ? c1 : k == 2 ? c2 : k == 3 ? c3 : k == 4 ? 0.0 : k == 5 ? -c3 :
           k == 6 ? -c2 : k == 7 ? -c1 : k == 8 ? -1.0 : k == 9 ? -c1 : k == 10 ? -c2 : k == 11 ? -c3 :
           k == 12 ? 0.0 : k == 13 ? c3 : k == 14 ? c2 : c1;
}
__host__ __device__ constexpr double sin16(int k) { return cos16(k - 4); }

// b * exp(DIR 2 pi i e / 16) with e a compile-time constant after unrolling;
// the four axis-aligned roots cost no multiply.
template <int DIR, typename T> __device__ __forceinline__ cplx<T> rot16(cplx<T> b, int e) {
    e &= 15;
    if (e == 0) return b;
    if (e == 8) return mk<T>(-b.x, -b.y);
    if (e == 4) return DIR > 0 ? mk<T>(-b.y, b.x) : mk<T>(b.y, -b.x);    // * (+-i)
    if (e == 12) return DIR > 0 ? mk<T>(b.y, -b.x) : mk<T>(-b.y, b.x);
    const T c = T(cos16(e)), s = T(DIR * sin16(e));
    return mk<T>(b.x * c - b.y * s, b.x * s + b.y * c);
}

__host__ __device__ constexpr int bitrev(int i, int n) {
    int r = 0;
    for (int b = 1; b < n; b <<= 1) { r = (r << 1) | (i & 1); i >>= 1; }
    return r;
}

// In-register DFT of size R (1, 2, 4, 8 or 16): X_k = sum_j v_j exp(DIR 2 pi i jk/R),
// natural order in and out; iterative radix-2 decimation in time.
template <int R, int DIR, typename T> __device__ __forceinline__ void dft_reg(cplx<T> *v) {
    if constexpr (R > 1) {
        cplx<T> w[R];
#pragma unroll
        for (int i = 0; i < R; ++i) w[bitrev(i, R)] = v[i];
#pragma unroll
        for (int len = 2; len <= R; len <<= 1) {
#pragma unroll
            for (int st = 0; st < R; st += len) {
#pragma unroll
                for (int m = 0; m < len / 2; ++m) {
                    const cplx<T> a = w[st + m];
                    const cplx<T> b = rot16<DIR, T>(w[st + m + len / 2], m * (16 / len));
                    w[st + m] = cadd<T>(a, b);
                    w[st + m + len / 2] = csub<T>(a, b);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < R; ++i) v[i] = w[i];
    }
}

// ---------------------------------------------------------------------------
// Batched length-N Stockham FFT.  A CTA runs F FFTs side by side; FFT f is
// served by TPF = N / E threads ("lanes"), each holding E = min(N, 16) values
// in registers.  On entry and on exit lane l holds positions l + TPF * e
// (e = 0..E-1) in natural order.  Passes exchange data through shared memory
// laid out as element (pos, f) at (pos + pos/16) * F + f: the one-slot pad per
// 16 positions keeps the stride-R writes of the first pass free of bank
// conflicts for F <= 16.
//
// Stockham radix-R pass with P = product of the radices already done:
// butterfly i (0 <= i < N/R) reads x[i + r N/R], multiplies by
// exp(DIR 2 pi i r k / (P R)) with k = i mod P, transforms over r, and writes
// y[(i / P) P R + k + r P].
// ---------------------------------------------------------------------------
constexpr int kTwiddleN = 1024;   // roots-of-unity table length (largest FFT)

template <int N> struct FftShape {
    static constexpr int E = N < 16 ? N : 16;
    static constexpr int TPF = N / E;
};

__device__ __forceinline__ int spad(int pos) { return pos + (pos >> 4); }

template <typename T, int N, int DIR, int P>
__device__ __forceinline__ void fft_passes(cplx<T> *v, int lane, cplx<T> *sbuf, int F, int f,
                                           const cplx<T> *__restrict__ tw) {
    constexpr int E = FftShape<N>::E, TPF = FftShape<N>::TPF;
    constexpr int REM = N / P;
    constexpr int R = REM >= 16 ? 16 : REM;
    constexpr bool LAST = (P * R == N);
    constexpr int BPT = E / R;                    // butterflies per thread
    static_assert(R >= 1 && E % R == 0, "radix must divide the values per thread");
    cplx<T> out[E];
#pragma unroll
    for (int s = 0; s < BPT; ++s) {
        const int i = lane + s * TPF;
        const int k = i & (P - 1);
        cplx<T> u[R];
#pragma unroll
        for (int r = 0; r < R; ++r) u[r] = v[s + r * BPT];
        if constexpr (P > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                // exp(DIR 2 pi i r k / (P R)) from the forward table exp(-2 pi i m / kTwiddleN)
                const int m = r * k * (kTwiddleN / (P * R));
                cplx<T> w = tw[m];
                if (DIR > 0) w.y = -w.y;
                u[r] = cmul<T>(u[r], w);
            }
        }
        dft_reg<R, DIR, T>(u);
#pragma unroll
        for (int r = 0; r < R; ++r) out[s + r * BPT] = u[r];
        if constexpr (!LAST) {
            const int j = (i / P) * P * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) sbuf[spad(j + r * P) * F + f] = u[r];
        }
    }
    if constexpr (LAST) {
        // positions i + r N/R = lane + TPF (s + r BPT): already the exit layout
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = out[e];
    } else {
        __syncthreads();
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = sbuf[spad(lane + TPF * e) * F + f];
        __syncthreads();
        fft_passes<T, N, DIR, P * R>(v, lane, sbuf, F, f, tw);
    }
}

// Full unnormalised FFT of the values held by this thread (see above).
// Every thread of the CTA must call it (it synchronises the CTA).
template <typename T, int N, int DIR>
__device__ __forceinline__ void fft(cplx<T> *v, int lane, cplx<T> *sbuf, int F, int f,
                                    const cplx<T> *__restrict__ tw) {
    if constexpr (N > 1) fft_passes<T, N, DIR, 1>(v, lane, sbuf, F, f, tw);
}

// shared-memory complex elements one FFT batch needs for its exchanges
__host__ __device__ constexpr int fft_smem_elems(int N, int F) { return (N + N / 16) * F; }

}  // namespace pss

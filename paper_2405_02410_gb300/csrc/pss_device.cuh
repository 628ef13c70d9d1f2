// pss_device.cuh -- device building blocks of the sm_103a pseudo-spectral step:
// complex arithmetic, the counter-based Philox4x32-10 generator, in-register
// radix-2/4/8/16/32 DFTs, the shared-memory Stockham pass that strings them into
// length-N FFTs (the F and F^-1 of Eq. cubicexample, arXiv:2405.02410), and
// the TMA bulk-copy / mbarrier helpers that stage tiles into shared memory.
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
// Products and sums that several kernels must round alike are written with
// explicit round-to-nearest intrinsics: the compiler never contracts them into
// fused multiply-adds of its own choosing, so two kernels that run the same
// formula give the same bits whatever code surrounds it.
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double fmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double fadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float ffma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double ffma(double a, double b, double c) { return __fma_rn(a, b, c); }

// a b = (a.x b.x - a.y b.y) + i (a.x b.y + a.y b.x): one product rounded, the other fused
template <typename T> __device__ __forceinline__ cplx<T> cmul(cplx<T> a, cplx<T> b) {
    return mk<T>(ffma(a.x, b.x, -fmul(a.y, b.y)), ffma(a.x, b.y, fmul(a.y, b.x)));
}
template <typename T> __device__ __forceinline__ cplx<T> cscale(cplx<T> a, T s) { return mk<T>(fmul(a.x, s), fmul(a.y, s)); }
// q^2 = qx^2 + qy^2 with the same rounding in every kernel
template <typename T> __device__ __forceinline__ T q2sum(T qx, T qy) { return ffma(qx, qx, fmul(qy, qy)); }

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC'11): ten rounds of two 32x32 -> 64-bit products with a
// Weyl-sequence key schedule.
// ---------------------------------------------------------------------------
struct u32x4 { uint32_t x, y, z, w; };

constexpr uint32_t kPhiloxMulA = 0xD2511F53u, kPhiloxMulB = 0xCD9E8D57u;
constexpr uint32_t kPhiloxWeylA = 0x9E3779B9u, kPhiloxWeylB = 0xBB67AE85u;

// one 32 x 32 -> 64-bit product gives both halves a round needs
__device__ __forceinline__ void mul_wide(uint32_t a, uint32_t b, uint32_t &hi, uint32_t &lo) {
    const uint64_t p = (uint64_t)a * (uint64_t)b;
    hi = (uint32_t)(p >> 32);
    lo = (uint32_t)p;
}

__device__ __forceinline__ u32x4 philox4x32_10(u32x4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        uint32_t hiA, loA, hiB, loB;
        mul_wide(kPhiloxMulA, c.x, hiA, loA);
        mul_wide(kPhiloxMulB, c.z, hiB, loB);
        c = u32x4{hiB ^ c.y ^ k0, loB, hiA ^ c.w ^ k1, loA};
        k0 += kPhiloxWeylA;
        k1 += kPhiloxWeylB;
    }
    return c;
}

// The ten round keys of one key (k + r W mod 2^32): a thread that draws many
// numbers under one key computes them once, and each round then costs two
// wide multiplies and two three-input XORs.
struct PhiloxKey { uint32_t k0[10], k1[10]; };

__device__ __forceinline__ PhiloxKey philox_key(uint32_t k0, uint32_t k1) {
    PhiloxKey K;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        K.k0[r] = k0 + (uint32_t)r * kPhiloxWeylA;
        K.k1[r] = k1 + (uint32_t)r * kPhiloxWeylB;
    }
    return K;
}

__device__ __forceinline__ u32x4 philox4x32_10(u32x4 c, const PhiloxKey &K) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        uint32_t hiA, loA, hiB, loB;
        mul_wide(kPhiloxMulA, c.x, hiA, loA);
        mul_wide(kPhiloxMulB, c.z, hiB, loB);
        c = u32x4{hiB ^ c.y ^ K.k0[round], loB, hiA ^ c.w ^ K.k1[round], loA};
    }
    return c;
}

// u = ((x >> 8) + 0.5) / 2^24: exact in float and double, strictly inside (0, 1)
template <typename T> __device__ __forceinline__ T uniform24(uint32_t x) {
    return (T(x >> 8) + T(0.5)) * T(5.9604644775390625e-08);
}

// square root and reciprocal: FP32 through the hardware approximations
// (about 2 ulp), FP64 correctly rounded
__device__ __forceinline__ float fast_sqrt(float x) { return x > 0.0f ? x * rsqrtf(x) : 0.0f; }
__device__ __forceinline__ double fast_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float fast_rcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double fast_rcp(double x) { return 1.0 / x; }

// Box-Muller pair.  FP32 uses the hardware log2 / sin / cos approximations
// (absolute error ~1e-6 on these arguments); FP64 uses the libdevice calls.
__device__ __forceinline__ void box_muller(float u0, float u1, float &n1, float &n2) {
    const float r = fast_sqrt(-2.0f * __logf(u0));
    float s, c;
    __sincosf(6.283185307179586f * u1, &s, &c);
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
// 32nd roots of unity: cos(2 pi k / 32) from the exact first-octant values
// (cos(j pi / 16), j = 0..8) by quadrant symmetry.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr double cos_oct(int j) {
    return j == 0 ? 1.0 : j == 1 ? 0.98078528040323044913 : j == 2 ? 0.92387953251128675613 :
           j == 3 ? 0.83146961230254523708 : j == 4 ? 0.70710678118654752440 : j == 5 ? 0.55557023301960222474 :
           j == 6 ? 0.38268343236508977173 : j == 7 ? 0.19509032201612826785 : 0.0;
}
__host__ __device__ constexpr double cos32(int k) {
    k &= 31;
    return k <= 8 ? cos_oct(k) : k <= 16 ? -cos_oct(16 - k) : k <= 24 ? -cos_oct(k - 16) : cos_oct(32 - k);
}
__host__ __device__ constexpr double sin32(int k) { return cos32(k - 8); }

// b * exp(DIR 2 pi i e / 32) with e a compile-time constant after unrolling;
// the four axis-aligned roots cost no multiply.
template <int DIR, typename T> __device__ __forceinline__ cplx<T> rot32(cplx<T> b, int e) {
    e &= 31;
    if (e == 0) return b;
    if (e == 16) return mk<T>(-b.x, -b.y);
    if (e == 8) return DIR > 0 ? mk<T>(-b.y, b.x) : mk<T>(b.y, -b.x);    // * (+-i)
    if (e == 24) return DIR > 0 ? mk<T>(b.y, -b.x) : mk<T>(-b.y, b.x);
    const T c = T(cos32(e)), s = T(DIR * sin32(e));
    return mk<T>(ffma(b.x, c, -fmul(b.y, s)), ffma(b.x, s, fmul(b.y, c)));
}

__host__ __device__ constexpr int bitrev(int i, int n) {
    int r = 0;
    for (int b = 1; b < n; b <<= 1) { r = (r << 1) | (i & 1); i >>= 1; }
    return r;
}

// In-register DFT of size R (1, 2, 4, 8, 16 or 32): X_k = sum_j v_j exp(DIR 2 pi i jk/R),
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
                    const cplx<T> b = rot32<DIR, T>(w[st + m + len / 2], m * (32 / len));
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
// Batched length-N Stockham FFT in shared memory.  A CTA runs several FFTs
// side by side; FFT f is served by TPF = N/E threads ("lanes"; one thread
// for N <= 16) and owns a contiguous buffer slice of SF elements in which
// position p lives at pos + pos/16 (one pad slot per 16 keeps the stride-R
// writes of a pass free of bank conflicts).  SF is chosen per thread mapping
// so that FFTs side by side fall in different banks too.
//
// Stockham radix-R pass with P = product of the radices already done:
// butterfly i (0 <= i < N/R) reads x[i + r N/R], multiplies by
// exp(DIR 2 pi i r k / (P R)) with k = i mod P, transforms over r, and writes
// y[(i / P) P R + k + r P].  N = E^m * RL: m radix-E passes (E = 8 or 16; the
// middle ones share one loop body), then one radix-RL pass.  The first pass reads through a source
// functor and the last pass writes through a sink functor, so that
// element-wise work (a power, a mask, a scale, a store to global memory)
// rides on the loads and stores the transform makes anyway.
// ---------------------------------------------------------------------------

template <int N, int EMAX> struct FftShape {
    static constexpr int E = fft_E(N, EMAX);    // values per thread and pass (the radix of the main passes)
    static constexpr int TPF = N / E;           // threads per FFT
    static constexpr int LOG = ilog2(N);
    static constexpr int LOGE = ilog2(E);
    // N = E^m * RL: radix-E passes, then a last pass of radix RL <= E (a
    // small radix last keeps every pass's shared-memory stores conflict-free)
    static constexpr int RL = N <= 1 ? 1 : (LOG % LOGE == 0 ? E : 1 << (LOG % LOGE));
    static constexpr int LOGRL = ilog2(RL);
};

__device__ __forceinline__ int spad(int pos) { return pos + (pos >> 4); }
__host__ __device__ constexpr int padded(int n) { return n + n / 16; }

// Buffer slice per FFT when consecutive threads are lanes of one FFT: the
// slices of FFTs sharing a half-warp (TPF < 16) start TPF banks apart.
__host__ __device__ constexpr int sf_lane_fastest(int n) { return n < 16 ? n + 1 : padded(n); }
// Buffer slice per FFT when consecutive threads belong to consecutive FFTs
// (F FFTs per CTA): slices start 16/F (F <= 16) or an odd number of elements apart.
__host__ __device__ constexpr int sf_fft_fastest(int n, int F) {
    const int m = F >= 16 ? 1 : 16 / F;
    const int s = padded(n) > 1 ? padded(n) : 1;
    return s + ((m - s % 16 + 16) % 16);
}

// Buffer slice per FFT for the row kernel: lane-fastest passes, and a
// split loop that reads 4 pairs side by side (slices 8 banks apart when a
// half-warp is a single FFT, N >= 256).
__host__ __device__ constexpr int sf_row(int n) {
    return n >= 256 ? padded(n) + ((4 - padded(n) % 16 + 16) % 16) : sf_lane_fastest(n);
}

template <typename T, int N, int EMAX, int R, int DIR, class Src, class Dst>
__device__ __forceinline__ void stockham_pass(Src src, Dst dst, int logP, int lane,
                                              const cplx<T> *__restrict__ tw) {
    constexpr int LOGR = R == 1 ? 0 : R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : 4;
    constexpr int TPF = FftShape<N, EMAX>::TPF;
    constexpr int STRIDE = N / R;
    constexpr int BPT = STRIDE / TPF;            // butterflies per thread
    const int P = 1 << logP;
#pragma unroll 1
    for (int s = 0; s < BPT; ++s) {
        const int i = lane + s * TPF;
        const int k = i & (P - 1);
        cplx<T> u[R];
#pragma unroll
        for (int r = 0; r < R; ++r) u[r] = src(i + r * STRIDE);
        if (P > 1) {
            // this pass's twiddles exp(-2 pi i r k / (P R)), stored [r - 1][k] from
            // entry P - E on; consecutive lanes read consecutive entries
            const cplx<T> *__restrict__ twp = tw + (P - FftShape<N, EMAX>::E) + k;
#pragma unroll
            for (int r = 1; r < R; ++r) {
                cplx<T> w = twp[(r - 1) * P];
                if (DIR > 0) w.y = -w.y;
                u[r] = cmul<T>(u[r], w);
            }
        }
        dft_reg<R, DIR, T>(u);
        const int j = ((i - k) << LOGR) + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dst(j + (r << logP), u[r]);
    }
}

// Full unnormalised FFT (DIR = -1 forward, +1 inverse) of the thread's FFT.
// src(p) gives input position p; the last pass hands (p, value, free) to
// sink, where `free` is this FFT's slice of the work buffer the last pass
// does not read (b0 or b1; the returned index says which).  b0, b1 are this
// FFT's slices; src may read b1 but never b0.  Every thread of the CTA must
// call it (it synchronises the CTA between passes); threads with
// active = false only take part in the barriers.
template <typename T, int N, int EMAX, int DIR, class Src, class Sink>
__device__ __forceinline__ int fft_run(Src src, Sink sink, cplx<T> *b0, cplx<T> *b1, int lane, bool active,
                                       const cplx<T> *__restrict__ tw) {
    using S = FftShape<N, EMAX>;
    if constexpr (N == 1) {
        if (active) sink(0, src(0), b0);
        return 0;
    } else if constexpr (S::LOG <= S::LOGE) {
        if (active) stockham_pass<T, N, EMAX, N, DIR>(src, [&](int p, cplx<T> v) { sink(p, v, b0); }, 0, lane, tw);
        return 0;
    } else {
        constexpr int E = S::E, LOGE = S::LOGE;
        if (active)
            stockham_pass<T, N, EMAX, E, DIR>(src, [&](int p, cplx<T> v) { b0[spad(p)] = v; }, 0, lane, tw);
        __syncthreads();
        cplx<T> *cur = b0, *nxt = b1;
        int which = 1;
        int logP = LOGE;
#pragma unroll 1
        for (; logP + S::LOGRL < S::LOG; logP += LOGE) {
            if (active)
                stockham_pass<T, N, EMAX, E, DIR>([&](int p) { return cur[spad(p)]; },
                                            [&](int p, cplx<T> v) { nxt[spad(p)] = v; }, logP, lane, tw);
            __syncthreads();
            cplx<T> *tmp = cur; cur = nxt; nxt = tmp;
            which ^= 1;
        }
        if (active)
            stockham_pass<T, N, EMAX, S::RL, DIR>([&](int p) { return cur[spad(p)]; },
                                                  [&](int p, cplx<T> v) { sink(p, v, nxt); }, logP, lane, tw);
        return which;
    }
}

// ---------------------------------------------------------------------------
// Programmatic dependent launch: a kernel launched with programmatic stream
// serialisation may start while its predecessor drains.  pdl_wait() blocks
// until the predecessor grid has completed and its writes are visible (a
// no-op without PDL); pdl_trigger() lets the successor launch.  Every kernel
// waits before touching data the previous kernel wrote and triggers only
// after that wait, so a successor's launch implies that every kernel before
// the current one has completed.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ---------------------------------------------------------------------------
// TMA bulk copies (cp.async.bulk, no tensor map) completing on an mbarrier.
// Every wait is bounded: after kWaitLimit polls the kernel records
// PSS_STATUS_TIMEOUT and takes its early exit.  A poll lets the hardware
// suspend the waiting thread for up to kWaitSuspendNs (it resumes as soon as
// the phase completes), so waiting warps leave the issue slots to the other
// CTAs of the SM instead of spinning; the total wait stays bounded (at most
// kWaitLimit x kWaitSuspendNs, about 2 s).
// ---------------------------------------------------------------------------
constexpr int kWaitLimit = 1 << 20;
constexpr uint32_t kWaitSuspendNs = 2000;
constexpr int kStatusNonFinite = 1;
constexpr int kStatusTimeout = 2;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// global -> shared bulk copy of `bytes` (multiple of 16; both addresses 16-byte aligned)
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// shared -> global bulk copy (bytes a multiple of 16; both addresses 16-byte
// aligned); the issuing thread commits and later waits for the group
__device__ __forceinline__ void bulk_s2g(void *dst, const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// generic-proxy shared-memory writes become visible to the bulk copy engine
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase), "r"(kWaitSuspendNs)
        : "memory");
    return ok != 0;
}

// The calling thread alone polls phase `phase` of `bar`, at most kWaitLimit
// times; false when the wait ran out.
__device__ __forceinline__ bool mbar_poll(uint64_t *bar, uint32_t phase) {
    for (int it = 0; it < kWaitLimit; ++it)
        if (mbar_try_wait(bar, phase)) return true;
    return false;
}

// All threads wait for phase `phase` of `bar` (at most `limit` polls each,
// 0: kWaitLimit).  Returns true for the whole CTA when the copies landed;
// false (for the whole CTA) when a bounded wait ran out, after a second
// bounded wait for the copies still in flight.
__device__ __forceinline__ bool mbar_wait_all(uint64_t *bar, uint32_t phase, int *status, int limit = kWaitLimit) {
    bool ok = false;
    if (limit <= 0) limit = kWaitLimit;
    for (int it = 0; it < limit && !ok; ++it) ok = mbar_try_wait(bar, phase);
    if (__syncthreads_and(ok)) return true;
    if (threadIdx.x == 0 && status) atomicOr(status, kStatusTimeout);
    for (int it = 0; it < limit && !ok; ++it) ok = mbar_try_wait(bar, phase);
    __syncthreads();
    return false;
}

}  // namespace pss

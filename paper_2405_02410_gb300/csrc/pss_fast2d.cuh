// pss_fast2d.cuh -- the FP32 2D step with one warp per transform
// (arXiv:2405.02410, section "What cuPSS calculates", Eq. timeupdate).
//
// For a 2D field whose sides are 256, 512 or 1024 points, every length-N
// transform of the step is run by a single warp in shared memory, so its
// passes meet at __syncwarp instead of CTA barriers.  Two kernels per step,
// with the same split of the work as the generic path:
//
//   k2_col (one CTA per tile of kTileW = 4 columns kx, all ky): the state,
//       the x-transformed product and the step's noise are staged with TMA;
//       four FFT groups (one per column) run the forward y-FFT; then every warp
//       updates the modes (Eq. timeupdate), the Hermitian part is taken on the
//       kx = 0, Nx/2 planes, the state goes back with one bulk copy and the FFT
//       groups transform the de-aliased, 1/N_sites-scaled kept columns back
//       along y.  Block 0 advances the step counter.
//   k2_row (one CTA per NW pairs of rows): group j takes rows r0 + 2j and
//       r0 + 2j + 1 as one complex transform (z = a + i b): C2R of the kept
//       columns, power p in real space, R2C, split into the two half spectra
//       (with real_out, the de-aliased real rows are stored too: the adjoint's
//       recomputed forward steps keep them).
//       Beside the transform groups, "noise" warps draw the Philox noise of the
//       next step (unit amplitude, tiled like the state) for the column kernel:
//       the generator has no data dependence, so it fills the issue slots the
//       latency-bound transforms leave idle.
//
// Only forward transforms are coded: an inverse is conj(F(conj(x))).  The
// column kernel stores the conjugate of its y-inverse (T1 = F(conj X)), which
// the row kernel's staging and split absorb, so no pass body exists twice.
// Each kernel runs its transforms from one inlined call site, and a pass
// loops over its butterflies: the code a kernel streams through an SM stays
// small (fully unrolled one-warp FFTs spent most of their time waiting for
// instruction fetch).
//
// The two work arrays between the kernels are column-major, [kx][y] with
// column kx contiguous: a column is one contiguous run for k2_col (one bulk
// copy per tile, conflict-free reads along y, coalesced stores), and the NW
// row pairs of a k2_row CTA are a 16 NW-byte run of every column.  The state
// keeps the tiled layout of every other kernel.
#pragma once

#include "pss_kernels.cuh"

namespace pss {

// A group FFT of length N with radix-E passes (E = 8, 16, or 32 for N = 1024)
// and a last pass of radix RL, run by TPF = N / E threads: whole warps that
// meet at a named barrier, one warp (__syncwarp), or half a warp (N = 256,
// E = 16: two groups per warp, each synchronising its own half).  A group's
// two buffers hold BUF = N + N / 2^PS points (room for the padded
// intermediate results) and sit WS apart (the extra 4 staggers neighbouring
// groups over the banks).
template <int N, int E_> struct GShape {
    static_assert(N == 256 || N == 512 || N == 1024, "group FFTs of 256, 512 or 1024 points");
    static_assert(E_ == 8 || E_ == 16 || (E_ == 32 && N == 1024), "radix-8, -16 or (1024 points) -32 passes");
    static constexpr int E = E_;
    static constexpr int TPF = N / E;
    static_assert((TPF % 32 == 0 && TPF <= 128) || TPF == 16, "half a warp or up to four warps per transform");
    static constexpr int LOG = ilog2(N), LOGE = ilog2(E);
    static constexpr int LOGRL = LOG % LOGE == 0 ? LOGE : LOG % LOGE;
    static constexpr int RL = 1 << LOGRL;
    static constexpr int NPASS = (LOG - LOGRL) / LOGE + 1;
    static constexpr int PS = E == 32 ? 5 : 4;     // one pad slot per 2^PS points
    static constexpr int BUF = N + (N >> PS);
    static constexpr int WS = 2 * BUF + 4;
    // the buffer that holds a transform's result: the first pass writes b0,
    // the passes alternate
    static constexpr int OUT = NPASS % 2 == 1 ? 0 : 1;
};

// the group's barrier: named barrier `id` (1..15) over its TPF threads
template <int TPF> __device__ __forceinline__ void group_sync(int id) {
    if constexpr (TPF == 16) {
        __syncwarp(0xFFFFu << (threadIdx.x & 16));   // this half of the warp
    } else if constexpr (TPF == 32) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(id), "n"(TPF) : "memory");
    }
}

// The AND of `pred` over the `nthreads` threads meeting at named barrier `id`
// (every one of them gets the same answer).
__device__ __forceinline__ bool bar_and(int id, int nthreads, bool pred) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(id), "r"(nthreads)
        : "memory");
    return r != 0;
}

// Intermediate pass results are padded: position p lives at p + p / 2^PS
// (one slot per 16 points, per 32 for radix-32 passes), which keeps the
// stride-R stores of a pass and the strided loads of the next free of bank
// conflicts, and which, with R and the pass strides known at compile time,
// folds into constant address offsets.  Inputs and outputs of a transform are
// in natural order.
template <int PS> __device__ __forceinline__ int padp(int p) { return p + (p >> PS); }

__device__ __forceinline__ float pow_p(float x, int p) { return p == 3 ? x * x * x : ipow<float>(x, p); }

// One forward Stockham pass of radix R after P = 2^logP points have been
// combined (the pass structure of the generic kernels, butterfly
// i = gl + TPF s): read x[i + r N/R], multiply by exp(-2 pi i r k / (P R)),
// k = i mod P, transform over r, write y[(i - k) R + k + r P].  tw is the
// (N, E) table; with power p > 0 (natural-order output only) an output
// x + i y is stored as x^p + i (-y)^p: for z' = conj(z) that is
// Re(z)^p + i Im(z)^p; with ra, rb set (natural-order output only) x and -y
// also go to ra[q], rb[q] (the real rows Re z, Im z themselves); with ma, mb
// set (natural-order output only, instead of the power) the output is
// p ma[q]^(p-1) x + i p mb[q]^(p-1) (-y), the adjoint's linearised power.
// VAR selects which of these the pass is compiled with (0 none, 1 power and
// real rows, 2 the linearised power), so each kernel carries only its own.
template <int N, int E, int R, bool TWID, bool PADIN, bool PADOUT, int VAR = 0>
__device__ __forceinline__ void fpass(const float2 *src, float2 *dst, int logP, int gl,
                                      const float2 *__restrict__ tw, int power, float *ra = nullptr,
                                      float *rb = nullptr, const float *ma = nullptr, const float *mb = nullptr) {
    constexpr int TPF = GShape<N, E>::TPF;
    constexpr int STRIDE = N / R, BPT = STRIDE / TPF, LOGR = ilog2(R);
    static_assert(STRIDE % TPF == 0, "every thread takes whole butterflies");
    const int P = 1 << logP;
    // a thread's butterflies of a small-radix pass (at most 16 values in all)
    // run unrolled, so that their loads and arithmetic overlap; larger passes
    // keep the loop rolled (code size)
    constexpr bool UNROLL = R * BPT <= 16;
#pragma unroll (UNROLL ? BPT : 1)
    for (int s = 0; s < BPT; ++s) {
        const int i = gl + TPF * s, k = i & (P - 1);
        float2 u[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int p = i + r * STRIDE;
            u[r] = src[PADIN ? padp<GShape<N, E>::PS>(p) : p];
        }
        if constexpr (TWID) {
            const float2 *__restrict__ twp = tw + (P - E) + k;
#pragma unroll
            for (int r = 1; r < R; ++r) u[r] = cmul<float>(u[r], twp[(r - 1) * P]);
        }
        dft_reg<R, -1, float>(u);
        const int j = ((i - k) << LOGR) + k;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int q = j + r * P;
            float2 v = u[r];
            if constexpr (!PADOUT && VAR == 1) {
                if (ra) {
                    ra[q] = v.x;
                    rb[q] = -v.y;
                }
                if (power > 0) v = mk<float>(pow_p(v.x, power), pow_p(-v.y, power));
            }
            if constexpr (!PADOUT && VAR == 2) {
                if (ma)
                    v = mk<float>(float(power) * ipow<float>(ma[q], power - 1) * v.x,
                                  float(power) * ipow<float>(mb[q], power - 1) * (-v.y));
            }
            dst[PADOUT ? padp<GShape<N, E>::PS>(q) : q] = v;
        }
    }
}

// Unnormalised forward FFT (exponent -2 pi i) of length N by a group of TPF
// threads (gl = 0..TPF-1, barrier `id`).  `in` holds the input in natural
// order and may be b1, never b0; the result, in natural order, lands in b0 or
// b1 (GShape::OUT).  b0 and b1 hold BUF points each.  The caller makes the
// input visible to the group before the call; the result is visible to the
// group on return.  power, ra, rb, ma, mb, VAR: see fpass (applied on the
// last pass).
template <int N, int E, int VAR = 0>
__device__ __forceinline__ float2 *fft_fwd_group(const float2 *in, float2 *b0, float2 *b1, int gl, int id,
                                                 const float2 *__restrict__ tw, int power, float *ra = nullptr,
                                                 float *rb = nullptr, const float *ma = nullptr,
                                                 const float *mb = nullptr) {
    using S = GShape<N, E>;
    fpass<N, E, E, false, false, true>(in, b0, 0, gl, tw, 0);
    group_sync<S::TPF>(id);
    float2 *cur = b0, *nxt = b1;
    int logP = S::LOGE;
#pragma unroll 1
    for (; logP + S::LOGRL < S::LOG; logP += S::LOGE) {
        fpass<N, E, E, true, true, true>(cur, nxt, logP, gl, tw, 0);
        group_sync<S::TPF>(id);
        float2 *tmp = cur;
        cur = nxt;
        nxt = tmp;
    }
    fpass<N, E, S::RL, true, true, false, VAR>(cur, nxt, logP, gl, tw, power, ra, rb, ma, mb);
    group_sync<S::TPF>(id);
    return nxt;
}

// The last pass of a group FFT with its natural-order outputs handed to
// sink(q, value) instead of stored (same butterflies and arithmetic as fpass).
template <int N, int E, int R, class Sink>
__device__ __forceinline__ void fpass_sink(const float2 *src, int logP, int gl, const float2 *__restrict__ tw,
                                           Sink &&sink) {
    constexpr int TPF = GShape<N, E>::TPF;
    constexpr int STRIDE = N / R, BPT = STRIDE / TPF, LOGR = ilog2(R);
    static_assert(STRIDE % TPF == 0, "every thread takes whole butterflies");
    const int P = 1 << logP;
    constexpr bool UNROLL = R * BPT <= 16;
#pragma unroll (UNROLL ? BPT : 1)
    for (int s = 0; s < BPT; ++s) {
        const int i = gl + TPF * s, k = i & (P - 1);
        float2 u[R];
#pragma unroll
        for (int r = 0; r < R; ++r) u[r] = src[padp<GShape<N, E>::PS>(i + r * STRIDE)];
        const float2 *__restrict__ twp = tw + (P - E) + k;
#pragma unroll
        for (int r = 1; r < R; ++r) u[r] = cmul<float>(u[r], twp[(r - 1) * P]);
        dft_reg<R, -1, float>(u);
        const int j = ((i - k) << LOGR) + k;
#pragma unroll
        for (int r = 0; r < R; ++r) sink(j + r * P, u[r]);
    }
}

// fft_fwd_group whose last pass hands each output to sink(q, value).  The
// input is in b1 (natural order); the last pass reads b1 when the transform
// has an odd number of passes, else b0, so the other buffer (SinkShape::FREE)
// is free for the sink to write.  No barrier follows the last pass.
template <int N, int E> struct SinkShape {
    static constexpr bool LAST_READS_B1 = (GShape<N, E>::NPASS - 1) % 2 == 0;
};
template <int N, int E, class Sink>
__device__ __forceinline__ void fft_fwd_group_sink(float2 *b0, float2 *b1, int gl, int id,
                                                   const float2 *__restrict__ tw, Sink &&sink) {
    using S = GShape<N, E>;
    static_assert(S::NPASS >= 2, "the sink pass reads padded intermediate results");
    {
        fpass<N, E, E, false, false, true>(b1, b0, 0, gl, tw, 0);
        group_sync<S::TPF>(id);
        float2 *cur = b0, *nxt = b1;
        int logP = S::LOGE;
#pragma unroll 1
        for (; logP + S::LOGRL < S::LOG; logP += S::LOGE) {
            fpass<N, E, E, true, true, true>(cur, nxt, logP, gl, tw, 0);
            group_sync<S::TPF>(id);
            float2 *tmp = cur;
            cur = nxt;
            nxt = tmp;
        }
        fpass_sink<N, E, S::RL>(cur, logP, gl, tw, sink);
    }
}

// ---- group FFTs with their first or last pass on registers ----------------
// Thread gl of a group takes input points gl + TPF m (m = 0..E-1) in the first
// pass of a transform, and the last pass leaves it with output points
// gl + TPF (s + BPT r) of its butterflies s and outputs r: the same set.  So
// a transform can start from values loaded from global memory, or from the
// outputs of the transform before it, without a round trip through shared
// memory: x[m] holds point gl + TPF m.  The butterflies and their arithmetic
// are those of fpass, so the results are the same bits.

// first pass (radix E, no twiddles) from x[] into dst (padded), as fpass<N, E, E, false, false, true>
template <int N, int E>
__device__ __forceinline__ void fpass_first_regs(float2 (&x)[E], float2 *dst, int gl) {
    using S = GShape<N, E>;
    dft_reg<E, -1, float>(x);
    const int j = gl << S::LOGE;
#pragma unroll
    for (int r = 0; r < E; ++r) dst[padp<S::PS>(j + r)] = x[r];
}

// the middle passes (radix E, twiddled, padded in and out) after the first
// pass wrote cur; on return cur is the buffer the last pass reads and nxt
// the other one.  Returns log2 of the points combined so far.
template <int N, int E>
__device__ __forceinline__ int fpass_middle(float2 *&cur, float2 *&nxt, int gl, int id,
                                            const float2 *__restrict__ tw) {
    using S = GShape<N, E>;
    int logP = S::LOGE;
#pragma unroll 1
    for (; logP + S::LOGRL < S::LOG; logP += S::LOGE) {
        fpass<N, E, E, true, true, true>(cur, nxt, logP, gl, tw, 0);
        group_sync<S::TPF>(id);
        float2 *tmp = cur;
        cur = nxt;
        nxt = tmp;
    }
    return logP;
}

// last pass (radix RL, twiddled) into x[]: x[m] = f(q, m, X_q), q = gl + TPF m
// (m a constant after unrolling: it may index the caller's register arrays)
template <int N, int E, class F>
__device__ __forceinline__ void fpass_last_regs_m(const float2 *src, int logP, int gl, const float2 *__restrict__ tw,
                                                  float2 (&x)[E], F &&f) {
    using S = GShape<N, E>;
    constexpr int R = S::RL, TPF = S::TPF, STRIDE = N / R, BPT = STRIDE / TPF, LOGR = ilog2(R);
    static_assert(BPT * R == E, "a thread's last-pass outputs are its first-pass inputs");
    const int P = 1 << logP;
#pragma unroll
    for (int s = 0; s < BPT; ++s) {
        const int i = gl + TPF * s, k = i & (P - 1);
        float2 u[R];
#pragma unroll
        for (int r = 0; r < R; ++r) u[r] = src[padp<S::PS>(i + r * STRIDE)];
        const float2 *__restrict__ twp = tw + (P - E) + k;
#pragma unroll
        for (int r = 1; r < R; ++r) u[r] = cmul<float>(u[r], twp[(r - 1) * P]);
        dft_reg<R, -1, float>(u);
        const int j = ((i - k) << LOGR) + k;
#pragma unroll
        for (int r = 0; r < R; ++r) x[s + BPT * r] = f(j + r * P, s + BPT * r, u[r]);
    }
}
// the same with x[m] = f(q, X_q)
template <int N, int E, class F>
__device__ __forceinline__ void fpass_last_regs(const float2 *src, int logP, int gl, const float2 *__restrict__ tw,
                                                float2 (&x)[E], F &&f) {
    fpass_last_regs_m<N, E>(src, logP, gl, tw, x, [&](int q, int, float2 v) { return f(q, v); });
}

// A group FFT from x[] (its first pass writes b0, which must be free) whose
// last pass hands its outputs to sink(q, value) (no barrier after it).
template <int N, int E, class Sink>
__device__ __forceinline__ void fft_regs_sink(float2 (&x)[E], float2 *b0, float2 *b1, int gl, int id,
                                              const float2 *__restrict__ tw, Sink &&sink) {
    fpass_first_regs<N, E>(x, b0, gl);
    group_sync<GShape<N, E>::TPF>(id);
    float2 *cur = b0, *nxt = b1;
    const int logP = fpass_middle<N, E>(cur, nxt, gl, id, tw);
    fpass_sink<N, E, GShape<N, E>::RL>(cur, logP, gl, tw, sink);
}

// A group FFT from x[] back into x[] (x[m] = f(q, X_q)); the last pass reads
// b1 when the transform has an odd number of passes, else b0 (no barrier after it).
template <int N, int E, class F>
__device__ __forceinline__ void fft_regs_regs(float2 (&x)[E], float2 *b0, float2 *b1, int gl, int id,
                                              const float2 *__restrict__ tw, F &&f) {
    fpass_first_regs<N, E>(x, b0, gl);
    group_sync<GShape<N, E>::TPF>(id);
    float2 *cur = b0, *nxt = b1;
    const int logP = fpass_middle<N, E>(cur, nxt, gl, id, tw);
    fpass_last_regs<N, E>(cur, logP, gl, tw, x, f);
}

// fft_regs_regs with x[m] = f(q, m, X_q)
template <int N, int E, class F>
__device__ __forceinline__ void fft_regs_regs_m(float2 (&x)[E], float2 *b0, float2 *b1, int gl, int id,
                                                const float2 *__restrict__ tw, F &&f) {
    fpass_first_regs<N, E>(x, b0, gl);
    group_sync<GShape<N, E>::TPF>(id);
    float2 *cur = b0, *nxt = b1;
    const int logP = fpass_middle<N, E>(cur, nxt, gl, id, tw);
    fpass_last_regs_m<N, E>(cur, logP, gl, tw, x, f);
}

// A group FFT of the natural-order input in b1 into x[] (x[m] = f(q, X_q));
// the last pass reads the same buffer as fft_regs_regs's (no barrier after it).
template <int N, int E, class F>
__device__ __forceinline__ void fft_smem_regs(float2 *b0, float2 *b1, int gl, int id, const float2 *__restrict__ tw,
                                              float2 (&x)[E], F &&f) {
    fpass<N, E, E, false, false, true>(b1, b0, 0, gl, tw, 0);
    group_sync<GShape<N, E>::TPF>(id);
    float2 *cur = b0, *nxt = b1;
    const int logP = fpass_middle<N, E>(cur, nxt, gl, id, tw);
    fpass_last_regs<N, E>(cur, logP, gl, tw, x, f);
}

// A group FFT from x[] (first pass into b0, which must be free) whose result,
// in natural order, is returned in one of the two buffers, visible to the group.
template <int N, int E>
__device__ __forceinline__ float2 *fft_regs_smem(float2 (&x)[E], float2 *b0, float2 *b1, int gl, int id,
                                                 const float2 *__restrict__ tw) {
    fpass_first_regs<N, E>(x, b0, gl);
    group_sync<GShape<N, E>::TPF>(id);
    float2 *cur = b0, *nxt = b1;
    const int logP = fpass_middle<N, E>(cur, nxt, gl, id, tw);
    fpass<N, E, GShape<N, E>::RL, true, true, false>(cur, nxt, logP, gl, tw, 0);
    group_sync<GShape<N, E>::TPF>(id);
    return nxt;
}

// ---------------------------------------------------------------------------
// k2_col: y transforms of one tile (4 columns) fused with the update.
// Threads: four FFT groups of TPF threads (group c = column c, barrier 1 + c),
// then helper warps that join the update.  Shared memory (bytes): mbarrier |
// roots of unity (N) | PHI: state chunk [pos][4] | XIN: product columns
// [c][pos] | XI: unit-amplitude noise [pos][4] | the four groups' buffer
// pairs.  A column's P lands in buffer OUT of its group; the update writes
// the conjugated inverse input into the other.
// ---------------------------------------------------------------------------
template <int N, int E> struct Col2Smem {
    using S = GShape<N, E>;
    static constexpr size_t TW = 128;
    static constexpr size_t PHI = TW + sizeof(float2) * N;
    static constexpr size_t XIN = PHI + sizeof(float2) * 4 * N;
    static constexpr size_t XI = XIN + sizeof(float2) * 4 * N;
    static constexpr size_t WBUF = XI + sizeof(float2) * 4 * N;
    static constexpr size_t BYTES = WBUF + sizeof(float2) * 4 * S::WS;
    static constexpr int POFS = S::OUT * S::BUF;   // P (after the forward transform)
    static constexpr int UOFS = S::BUF - POFS;     // the inverse's (conjugated) input
};

template <int N, int E>
__global__ void __launch_bounds__(E == 8 ? 1024 : E == 16 ? 768 : 512, 1) k2_col(const ColArgs<float> a) {
    using C = float2;
    using S = GShape<N, E>;
    using L = Col2Smem<N, E>;
    constexpr int TPF = S::TPF, NF = 4 * TPF;   // FFT threads of the CTA
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);
    C *TW = reinterpret_cast<C *>(smem_raw + L::TW);
    C *PHI = reinterpret_cast<C *>(smem_raw + L::PHI);
    C *XIN = reinterpret_cast<C *>(smem_raw + L::XIN);
    C *XI = reinterpret_cast<C *>(smem_raw + L::XI);
    C *WBUF = reinterpret_cast<C *>(smem_raw + L::WBUF);
    __shared__ FieldP<float> sfp;
    const SysP<float> &sp = a.sp;
    const FieldP<float> &fp = sfp;
    const int t = threadIdx.x, nthr = blockDim.x;
    const int g = t / TPF, gl = t - g * TPF;                                        // FFT group (column) and its thread
    const int slot = a.slot0 + blockIdx.y;
    const size_t sofs = (size_t)slot * a.slot_stride + (size_t)blockIdx.x * 4 * N;   // the tile's chunk / columns
    const int kxt = blockIdx.x * 4;                                                  // first kx of the tile
    const bool step_mode = a.mode == COL_STEP;
    const bool with_noise = step_mode && a.noise != nullptr;
    const uint32_t chunk = (uint32_t)(4 * N * sizeof(C));
    // what no earlier kernel writes (roots of unity, parameters) is fetched
    // before the wait on the previous launch, so that with programmatic
    // dependent launch it overlaps that launch's tail
    if (t == 0) {
        mbar_init(bar, 1);
        mbar_expect_tx(bar, (uint32_t)(N * sizeof(C)) + chunk * (step_mode ? (with_noise ? 3u : 2u) : 1u));
        bulk_g2s(TW, a.tw + twiddle_offset(N, E), (uint32_t)(N * sizeof(C)), bar);
    }
    static_assert(sizeof(FieldP<float>) % 4 == 0, "FieldP is copied as 32-bit words");
    for (int i = t; i < (int)(sizeof(FieldP<float>) / 4); i += (int)blockDim.x)   // CTAs may be smaller than FieldP
        reinterpret_cast<uint32_t *>(&sfp)[i] = reinterpret_cast<const uint32_t *>(&a.fps[slot])[i];
    pdl_wait();
    pdl_trigger();
    if (t == 0) {
        bulk_g2s(PHI, a.state + sofs, chunk, bar);
        if (step_mode) bulk_g2s(XIN, a.in + sofs, chunk, bar);
        if (with_noise) bulk_g2s(XI, a.noise + sofs, chunk, bar);
    }
    __syncthreads();   // the barrier is initialised, the parameters are in place
    const bool ok = mbar_poll(bar, 0);

    const int kmx = fp.kmax[0], kmy = fp.kmax[1];
    const float scale = sp.inv_nsites;
    C *gb = WBUF + (g & 3) * S::WS;
    // Two transform phases from one call site: 0 = forward of the product
    // column (step mode), 1 = inverse of the kept column, stored conjugated.
#pragma unroll 1
    for (int ph = 0; ph < 2; ++ph) {
        const bool run = t < NF && (ph == 0 ? step_mode : kxt + g <= kmx);
        if (run) {
            const C *src = ph == 0 ? XIN + g * N : gb + L::UOFS;
            C *o = fft_fwd_group<N, E>(src, ph == 0 ? gb : gb + L::POFS, ph == 0 ? gb + S::BUF : gb + L::UOFS, gl,
                                       1 + g, TW, 0);
            if (ph == 1) {
                C *__restrict__ dst = a.out + sofs + (size_t)g * N;
#pragma unroll 4
                for (int p = gl; p < N; p += TPF) dst[p] = o[p];
            }
        }
        if (ph == 1) break;
        if (!__syncthreads_and(ok)) {
            if (t == 0 && a.d_status) atomicOr(a.d_status, kStatusTimeout);
            mbar_poll(bar, 0);   // copies still in flight land before the CTA's shared memory is released
            __syncthreads();
            return;
        }
        if (step_mode) {
            // ---- update (Eq. timeupdate) of every mode, two neighbouring columns
            // per thread and position, two positions in flight per thread
            float dtO[kPolyTerms], dtM[kPolyTerms];
#pragma unroll
            for (int i = 0; i < kPolyTerms; ++i) {
                dtO[i] = sp.dt * fp.O[i];
                dtM[i] = sp.dt * fp.M[i];
            }
            const bool has_product = fp.power > 0, noisy = with_noise && fp.noisy != 0;
            const float sigma0 = fp.sigma0;
            bool bad = false;
#pragma unroll 1
            for (int i0 = t; i0 < 2 * N; i0 += 2 * nthr) {
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int i = i0 + u * nthr;
                    if (i >= 2 * N) break;
                    const int pos = i >> 1, c0 = 2 * (i & 1), kx0 = kxt + c0;
                    C f0, f1, x0 = mk<float>(0.f, 0.f), x1 = x0;
                    ld_pair<float>(PHI + 4 * pos + c0, f0, f1);
                    if (noisy) {
                        ld_pair<float>(XI + 4 * pos + c0, x0, x1);
                        x0 = cscale<float>(x0, sigma0);
                        x1 = cscale<float>(x1, sigma0);
                    }
                    C *B0 = WBUF + c0 * S::WS;
                    C v0 = B0[L::POFS + pos], v1 = B0[S::WS + L::POFS + pos];
                    const float qy = fmul(float(signed_k(pos, N)), sp.gy);
                    const float qx0 = fmul(float(kx0), sp.gx), qx1 = fmul(float(kx0 + 1), sp.gx);
                    const float q2a = q2sum(qx0, qy), q2b = q2sum(qx1, qy);
                    v0 = update_mode<float>(f0, v0, x0, q2a, dtO, dtM, has_product);
                    v1 = update_mode<float>(f1, v1, x1, q2b, dtO, dtM, has_product);
                    if (kx0 >= sp.hx) v0 = mk<float>(0.f, 0.f);
                    if (kx0 + 1 >= sp.hx) v1 = mk<float>(0.f, 0.f);
                    bad |= !(fabsf(v0.x) + fabsf(v0.y) + fabsf(v1.x) + fabsf(v1.y) <= 3.0e38f);
                    st_pair<float>(PHI + 4 * pos + c0, v0, v1);
                    const bool ky_keep = abs(signed_k(pos, N)) <= kmy;
                    const float s0 = (ky_keep && kx0 <= kmx) ? scale : 0.f;
                    const float s1 = (ky_keep && kx0 + 1 <= kmx) ? scale : 0.f;
                    B0[L::UOFS + pos] = mk<float>(v0.x * s0, -v0.y * s0);
                    B0[S::WS + L::UOFS + pos] = mk<float>(v1.x * s1, -v1.y * s1);
                }
            }
            if (bad && a.d_status) atomicOr(a.d_status, kStatusNonFinite);
            __syncthreads();
            // Hermitian part on the kx = 0 and kx = Nx/2 planes (the field is
            // real): phi(kx, ky) <- (phi(kx, ky) + conj phi(kx, -ky)) / 2
            const int kh = sp.nx / 2;
            const int npl = (kxt == 0 ? 1 : 0) + ((kh >> 2) == (int)blockIdx.x ? 1 : 0);
            if (npl > 0) {
                const int cA = kxt == 0 ? 0 : (kh & 3), cB = kh & 3;
                constexpr int HALF = N / 2 + 1;
#pragma unroll 1
                for (int i = t; i < npl * HALF; i += nthr) {
                    const int j = i >= HALF ? 1 : 0, pos = i - j * HALF;
                    const int c = j ? cB : cA;
                    const int ppos = (N - pos) & (N - 1);
                    const C u0 = PHI[4 * pos + c], u1 = PHI[4 * ppos + c];
                    const C h = mk<float>(0.5f * (u0.x + u1.x), 0.5f * (u0.y - u1.y));
                    PHI[4 * pos + c] = h;
                    PHI[4 * ppos + c] = mk<float>(h.x, -h.y);
                    const bool kxk = kxt + c <= kmx;
                    C *U = WBUF + c * S::WS + L::UOFS;
                    const float s0 = (kxk && abs(signed_k(pos, N)) <= kmy) ? scale : 0.f;
                    const float s1 = (kxk && abs(signed_k(ppos, N)) <= kmy) ? scale : 0.f;
                    U[pos] = mk<float>(h.x * s0, -h.y * s0);   // conj(h)
                    U[ppos] = mk<float>(h.x * s1, h.y * s1);   // conj(conj(h))
                }
            }
            // the state goes back with one bulk copy (its chunk is contiguous)
            fence_proxy_async();
            __syncthreads();
            if (t == 0) {
                C *sdst = a.state_out ? a.state_out : a.state;
                bulk_s2g(sdst + sofs, PHI, chunk);
                bulk_commit();
            }
        } else {
            // start of a run: the inverse input is the de-aliased, scaled state
#pragma unroll 1
            for (int i = t; i < 4 * N; i += nthr) {
                const int pos = i >> 2, c = i & 3;
                const float sc = (kxt + c <= kmx && abs(signed_k(pos, N)) <= kmy) ? scale : 0.f;
                const C v = PHI[i];
                WBUF[c * S::WS + L::UOFS + pos] = mk<float>(v.x * sc, -v.y * sc);
            }
            __syncthreads();
        }
    }
    if (step_mode && t == 0) {
        bulk_wait_read();   // PHI outlives the state write-back
        if (blockIdx.x == 0 && blockIdx.y == 0) *a.d_step += 1;   // no CTA of this kernel reads it
    }
}

// ---------------------------------------------------------------------------
// k2_row: x transforms of NW = a.G pairs of rows, group j (barrier 1 + j) on
// rows r0 + 2j, r0 + 2j + 1, then the noise warps.  The transform threads
// meet at barrier 15.  Shared memory: mbarrier | roots of unity (N) | per
// group two buffers of BUF points, WS apart.
//
// TILED = false: the 2D step's column-major work arrays, the input holding
// the conjugated y-inverse.  TILED = true: the tiled arrays of the generic
// kernels ([tile][row][4], input as it is), as the x pass of the 3D step and
// of the 2D adjoint step (mode ROW_ADJ: C2R of all columns, times
// p r^(p-1) with r the stored real rows, R2C); the CTA's rows of one tile are
// a 64 NW-byte run, moved as 16-byte pieces.
// ---------------------------------------------------------------------------
// A row group's buffer pair: WS apart in the 2D mapping (element (k, pair j)
// by consecutive threads: the extra 4 of WS puts the four pairs of a
// half-warp on distinct banks), WST apart plus a shift in the tiled mapping
// (element (tile, pair j): a half-warp covers 8 pairs of 2 tiles, 4 columns
// apart; the shifts (j & 3) + 8 ((j >> 2) & 1) spread them over all 16 bank
// pairs).
template <int N, int E> struct Row2Smem {
    static constexpr int WST = 2 * GShape<N, E>::BUF + 16;
    __host__ __device__ static size_t bytes(int nw, bool tiled) {
        return 128 + sizeof(float2) * ((size_t)N + (size_t)nw * (tiled ? WST : GShape<N, E>::WS));
    }
    __device__ static int base(int j, bool tiled) {
        return tiled ? j * WST + (j & 3) + 8 * ((j >> 2) & 1) : j * GShape<N, E>::WS;
    }
};

// Unit-amplitude noise (sigma0 = 1) of pairs q0, q0 + stride, ... < q1 of one
// slot, step `step`; pair q = (tile ny + pos) 2 + cp covers columns
// 4 tile + 2 cp, 4 tile + 2 cp + 1 at ky = pos and is stored as 16 bytes at
// element 2 q of the slot's tiled array.  Two pairs in flight per thread.
__device__ __forceinline__ void noise_range(const SysP<float> &sp, const FieldP<float> &fp, uint32_t step,
                                            float2 *__restrict__ out, int q0, int q1, int stride) {
    const int logny = __ffs(sp.ny) - 1;
    const PhiloxKey key = philox_key(fp.seed_lo, fp.seed_hi);
#pragma unroll 1
    for (int qa = q0; qa < q1; qa += 2 * stride) {
        float2 xa[2], xb[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int q = qa + u * stride;
            const int rest = q >> 1, pos = rest & (sp.ny - 1), kx0 = ((rest >> logny) << 2) + 2 * (q & 1);
            xa[u] = mk<float>(0.f, 0.f);
            xb[u] = xa[u];
            if (q < q1 && kx0 < sp.hx) {
                const float qy = fmul(float(signed_k(pos, sp.ny)), sp.gy);
                const float qx0 = fmul(float(kx0), sp.gx), qx1 = fmul(float(kx0 + 1), sp.gx);
                const float q2a = q2sum(qx0, qy), q2b = q2sum(qx1, qy);
                noise_pair<float>(kx0 == 0 || 2 * kx0 == sp.nx, kx0, pos, 0, noise_amp<float>(1.f, fp.noise_pow, q2a),
                                  noise_amp<float>(1.f, fp.noise_pow, q2b), kx0 + 1 < sp.hx, sp, (uint32_t)fp.field_id,
                                  key, step, xa[u], xb[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int q = qa + u * stride;
            if (q < q1) st_pair<float>(out + 2 * (size_t)q, xa[u], xb[u]);
        }
    }
}

template <int N, int E, bool TILED, bool ADJ>
__global__ void __launch_bounds__(E == 32 || TILED ? 512 : 1024) k2_row(const RowArgs<float> a) {
    using C = float2;
    using S = GShape<N, E>;
    constexpr int TPF = S::TPF;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);
    C *TW = reinterpret_cast<C *>(smem_raw + 128);
    C *WBUF = TW + N;
    const SysP<float> &sp = a.sp;
    const int NW = a.G, logNW = __ffs(NW) - 1;   // NW a power of two
    const int nf = NW * TPF;                     // transform threads
    const int t = threadIdx.x;
    const int g = t / TPF, gl = t - g * TPF;
    const int slot = a.slot0 + blockIdx.y;
    const int rows = sp.rows;
    const int r0 = blockIdx.x * 2 * NW;                                                  // first row of the CTA
    const size_t sofs = (size_t)slot * a.slot_stride + (size_t)r0 * (TILED ? 4 : 1);
    constexpr int H = N / 2 + 1;
    const int nrow_cta = (int)gridDim.x - a.noise_ctas;
    const bool noise_thread = (int)blockIdx.x >= nrow_cta || t >= nf;
    // roots of unity: one bulk copy, issued before the wait on the previous
    // launch (no kernel writes them) and in flight while the rows are loaded
    if (!noise_thread && t == 0) {
        mbar_init(bar, 1);
        mbar_expect_tx(bar, (uint32_t)(N * sizeof(C)));
        bulk_g2s(TW, a.tw + twiddle_offset(N, E), (uint32_t)(N * sizeof(C)), bar);
    }
    pdl_wait();
    pdl_trigger();
    // ---- noise: the next step's, split between the extra noise CTAs (the
    // first noise_share/64 of the pairs, every thread) and the noise warps of
    // the row CTAs (the rest)
    if (noise_thread) {
        const FieldP<float> &fp = a.fps[slot];
        if (a.noise && fp.noisy) {
            const int Q = sp.ntiles * sp.ny * 2;
            const int Qn = a.noise_ctas > 0 ? (int)((long long)Q * a.noise_share / 64) : 0;
            int q0, q1, i, n;
            if ((int)blockIdx.x >= nrow_cta) {
                const int b = blockIdx.x - nrow_cta;
                q0 = (int)((long long)Qn * b / a.noise_ctas);
                q1 = (int)((long long)Qn * (b + 1) / a.noise_ctas);
                i = t;
                n = blockDim.x;
            } else {
                const int b = blockIdx.x;
                q0 = Qn + (int)((long long)(Q - Qn) * b / nrow_cta);
                q1 = Qn + (int)((long long)(Q - Qn) * (b + 1) / nrow_cta);
                i = t - nf;
                n = (int)blockDim.x - nf;
            }
            if (n > 0) noise_range(sp, fp, (uint32_t)(*a.d_step), a.noise + (size_t)slot * a.slot_stride, q0 + i, q1, n);
        }
        return;
    }
    // ---- stage Y = conj(Z), Z_k = A_k + i B_k (k <= N/2), conj(A_{N-k}) +
    // i conj(B_{N-k}) above, into the second buffer of group j.  With
    // (ar, ai, br, bi) the values of rows r0 + 2j, r0 + 2j + 1 at column k:
    // Y_k = (ar - bi, -ai - br), Y_{N-k} = (ar + bi, ai - br) for the values
    // as they are (TILED), and the two swapped when the input holds their
    // conjugates (the 2D path).  All of a thread's loads are issued before the
    // first use.
    constexpr bool adj = TILED && ADJ;   // mode ROW_ADJ
    // ROW_ADJ: the real rows r0 .. r0 + 2 NW - 1 (one contiguous run), which the
    // first transform's last pass multiplies in, go to shared memory behind the
    // group buffers now, all of a thread's loads in flight together, instead of
    // being read from global memory inside that pass
    float *MS = nullptr;
    if constexpr (adj) {
        MS = reinterpret_cast<float *>(smem_raw + Row2Smem<N, E>::bytes(NW, true));
        constexpr int PER = N / (2 * TPF), CH = PER < 4 ? PER : 4;   // float4 per thread, per batch of loads
        static_assert(PER % CH == 0, "whole batches");
        const float4 *__restrict__ src =
            reinterpret_cast<const float4 *>(a.real_in + (size_t)slot * a.real_stride + (size_t)r0 * N);
        float4 *ms4 = reinterpret_cast<float4 *>(MS);
#pragma unroll 1
        for (int p0 = 0; p0 < PER; p0 += CH) {
            float4 v[CH];
#pragma unroll
            for (int c = 0; c < CH; ++c) v[c] = __ldcg(src + t + (p0 + c) * nf);
#pragma unroll
            for (int c = 0; c < CH; ++c) ms4[t + (p0 + c) * nf] = v[c];
        }
    }
    const int kcm = adj ? sp.hx : a.kx_cols_max;
    const int kc = adj ? sp.hx : a.fps[slot].kx_cols;
    auto stage = [&](int k, int j, float ar, float ai, float br, float bi) {
        C *Y = WBUF + Row2Smem<N, E>::base(j, TILED) + S::BUF;
        if (k >= kc) { ar = 0.f; ai = 0.f; br = 0.f; bi = 0.f; }
        if (k == 0 || k == N / 2) { ai = 0.f; bi = 0.f; }   // the half spectra of real rows
        const C lo = mk<float>(ar - bi, -ai - br), hi = mk<float>(ar + bi, ai - br);
        Y[k] = TILED ? lo : hi;
        if (k > 0 && k < N / 2) Y[N - k] = TILED ? hi : lo;
    };
    if constexpr (!TILED) {
        const C *__restrict__ in = a.in + sofs;
        const int total = H << logNW;
#pragma unroll 1
        for (int base = 0; base < total; base += 8 * nf) {
            float4 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int idx = base + u * nf + t;
                const int k = idx >> logNW;
                v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (idx < total && k < kcm)
                    v[u] = __ldcg(reinterpret_cast<const float4 *>(in + (size_t)k * rows + 2 * (idx & (NW - 1))));
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int idx = base + u * nf + t;
                if (idx >= total) break;
                stage(idx >> logNW, idx & (NW - 1), v[u].x, v[u].y, v[u].z, v[u].w);
            }
        }
    } else {
        // item (tile, pair j): the 64 bytes of rows r0 + 2j, r0 + 2j + 1 of the tile
        const float4 *__restrict__ in = reinterpret_cast<const float4 *>(a.in + sofs);
        const int ntl = (kcm + 3) >> 2;
        const int total = ntl << logNW;
#pragma unroll 1
        for (int base = 0; base < total; base += 2 * nf) {
            float4 v[2][4];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int idx = base + u * nf + t;
                const float4 *p = in + ((size_t)(idx >> logNW) * rows + 2 * (idx & (NW - 1))) * 2;
#pragma unroll
                for (int q = 0; q < 4; ++q) v[u][q] = idx < total ? __ldcg(p + q) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int idx = base + u * nf + t;
                if (idx >= total) break;
                const int k0 = (idx >> logNW) << 2, j = idx & (NW - 1);
                // row a: (c0, c1) (c2, c3) in v[0], v[1]; row b in v[2], v[3]
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float4 va = v[u][c >> 1], vb = v[u][2 + (c >> 1)];
                    if (k0 + c <= N / 2)
                        stage(k0 + c, j, (c & 1) ? va.z : va.x, (c & 1) ? va.w : va.y, (c & 1) ? vb.z : vb.x,
                              (c & 1) ? vb.w : vb.y);
                }
            }
        }
        // the columns past the staged tiles are zero
        const int kz = ntl << 2, nz = H - kz;
        for (int idx = t; idx < (nz > 0 ? nz << logNW : 0); idx += nf)
            stage(kz + (idx >> logNW), idx & (NW - 1), 0.f, 0.f, 0.f, 0.f);
    }
    const int power = a.fps[slot].power;
    asm volatile("bar.sync 15, %0;" ::"r"(nf) : "memory");   // the mbarrier is initialised; Y is staged
    if (!bar_and(15, nf, mbar_poll(bar, 0))) {
        // the copy did not land in time: record it, wait (bounded) for it and leave together
        if (t == 0 && a.d_status) atomicOr(a.d_status, kStatusTimeout);
        mbar_poll(bar, 0);
        return;
    }
    // ---- z' = F(Y) = conj(z) = a - i b; its last pass forms u = a^p + i b^p,
    // the product of both rows (ROW_ADJ: p a^(p-1) Re z' + i p b^(p-1) (-Im z'),
    // with the stored real rows a, b), and stores the rows a and b themselves
    // when real_out is set; then W = F(u).  With radix-8 and radix-32 passes u
    // goes to W's first pass in registers and W lands in the group's first
    // buffer; the radix-16 kernels (64 registers per thread at 1024 threads)
    // pass u through shared memory and W lands in the second buffer.
    constexpr bool CHAIN = E != 16 || TILED;
    if constexpr (!CHAIN) {
        C *b0 = WBUF + Row2Smem<N, E>::base(g, TILED), *b1 = b0 + S::BUF;
        const C *src = b1;
        C *p0 = b0, *p1 = b1;
        float *ra = nullptr, *rb = nullptr;
        const float *ma = nullptr, *mb = nullptr;
        if (!TILED && a.real_out) {
            ra = a.real_out + (size_t)slot * a.real_stride + (size_t)(r0 + 2 * g) * N;
            rb = ra + N;
        }
        if (adj) {
            ma = MS + (size_t)(2 * g) * N;
            mb = ma + N;
        }
#pragma unroll 1
        for (int it = 0; it < 2; ++it) {
            C *o = fft_fwd_group<N, E, adj ? 2 : 1>(src, p0, p1, gl, 1 + g, TW, it == 0 ? power : 0,
                                                    it == 0 ? ra : nullptr, it == 0 ? rb : nullptr,
                                                    it == 0 ? ma : nullptr, it == 0 ? mb : nullptr);
            src = o;
            p0 = o == b0 ? b1 : b0;
            p1 = o;
        }
    } else {
        C *b0 = WBUF + Row2Smem<N, E>::base(g, TILED), *b1 = b0 + S::BUF;
        float *ra = nullptr, *rb = nullptr;
        const float *ma = nullptr, *mb = nullptr;
        if (!TILED && a.real_out) {
            ra = a.real_out + (size_t)slot * a.real_stride + (size_t)(r0 + 2 * g) * N;
            rb = ra + N;
        }
        if (adj) {
            ma = MS + (size_t)(2 * g) * N;
            mb = ma + N;
        }
        C x[E];
        fft_smem_regs<N, E>(b0, b1, gl, 1 + g, TW, x, [&](int q, C v) {
            if constexpr (adj) {
                v = mk<float>(float(power) * ipow<float>(ma[q], power - 1) * v.x,
                              float(power) * ipow<float>(mb[q], power - 1) * (-v.y));
            } else {
                if (ra) {
                    ra[q] = v.x;
                    rb[q] = -v.y;
                }
                if (power > 0) v = mk<float>(pow_p(v.x, power), pow_p(-v.y, power));
            }
            return v;
        });
        // the R2C's first pass writes the buffer the C2R's last pass did not read;
        // with either pass count the result is in b0
        constexpr bool LB1 = SinkShape<N, E>::LAST_READS_B1;
        fft_regs_smem<N, E>(x, LB1 ? b0 : b1, LB1 ? b1 : b0, gl, 1 + g, TW);
    }
    asm volatile("bar.sync 15, %0;" ::"r"(nf) : "memory");
    // ---- split into the half spectra of the two rows:
    // A_k = (W_k + conj W_{N-k}) / 2, B_k = (W_k - conj W_{N-k}) / 2i
    auto split = [&](int k, int j) {
        const C *Wj = WBUF + Row2Smem<N, E>::base(j, TILED) + (CHAIN ? 0 : S::BUF);
        const C wk = Wj[k], wm = Wj[(N - k) & (N - 1)];
        return make_float4(0.5f * (wk.x + wm.x), 0.5f * (wk.y - wm.y), 0.5f * (wk.y + wm.y), -0.5f * (wk.x - wm.x));
    };
    if constexpr (!TILED) {
        // (k, pair j) stored as 16 bytes
        C *__restrict__ out = a.out + sofs;
        const int total = H << logNW;
#pragma unroll 1
        for (int idx = t; idx < total; idx += nf) {
            const int k = idx >> logNW, j = idx & (NW - 1);
            *reinterpret_cast<float4 *>(out + (size_t)k * rows + 2 * j) = split(k, j);
        }
    } else {
        // (tile, pair j) stored as the 64 bytes of its two rows (zero past Nx/2)
        float4 *__restrict__ out = reinterpret_cast<float4 *>(a.out + sofs);
        const int total = sp.ntiles << logNW;
#pragma unroll 1
        for (int idx = t; idx < total; idx += nf) {
            const int k0 = (idx >> logNW) << 2, j = idx & (NW - 1);
            float4 ab[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) ab[c] = k0 + c <= N / 2 ? split(k0 + c, j) : make_float4(0.f, 0.f, 0.f, 0.f);
            float4 *p = out + ((size_t)(idx >> logNW) * rows + 2 * j) * 2;
            p[0] = make_float4(ab[0].x, ab[0].y, ab[1].x, ab[1].y);   // row a
            p[1] = make_float4(ab[2].x, ab[2].y, ab[3].x, ab[3].y);
            p[2] = make_float4(ab[0].z, ab[0].w, ab[1].z, ab[1].w);   // row b
            p[3] = make_float4(ab[2].z, ab[2].w, ab[3].z, ab[3].w);
        }
    }
}

// ---------------------------------------------------------------------------
// launchers: E is the radix of the FFT passes (8 or 16; 8 only for N = 256)
// ---------------------------------------------------------------------------
template <int N, int E> cudaError_t launch_col2_ne(const ColArgs<float> &a, int nslots, int ntiles, cudaStream_t st) {
    const int threads = 4 * GShape<N, E>::TPF + 32 * a.aux_warps;
    if (a.aux_warps < 1 || threads > (E == 8 ? 1024 : E == 16 ? 768 : 512)) return cudaErrorInvalidConfiguration;
    cudaError_t e = ensure_smem(k2_col<N, E>, Col2Smem<N, E>::BYTES);
    if (e != cudaSuccess) return e;
    return launch_pdl(k2_col<N, E>, dim3(ntiles, nslots), threads, Col2Smem<N, E>::BYTES, st, a);
}

template <int N, int E, bool TILED, bool ADJ>
cudaError_t launch_row2_ne(const RowArgs<float> &a, int nslots, cudaStream_t st) {
    const int nw = a.G, threads = nw * GShape<N, E>::TPF + 32 * a.noise_warps;
    if (nw < 1 || nw > 8 || (nw & (nw - 1)) || a.sp.rows % (2 * nw) || a.noise_warps < 0 ||
        threads > (E == 32 || TILED ? 512 : 1024) || (TILED && a.noise) || a.noise_ctas < 0 ||
        (a.noise_ctas > 0 && !a.noise) || a.noise_share < 0 || a.noise_share > 64)
        return cudaErrorInvalidConfiguration;
    // ROW_ADJ also stages the CTA's 2 nw real rows
    const size_t smem = Row2Smem<N, E>::bytes(nw, TILED) + (TILED && ADJ ? sizeof(float) * 2 * nw * N : 0);
    cudaError_t e = ensure_smem(k2_row<N, E, TILED, ADJ>, smem);
    if (e != cudaSuccess) return e;
    return launch_pdl(k2_row<N, E, TILED, ADJ>, dim3(a.sp.rows / (2 * nw) + a.noise_ctas, nslots), threads, smem,
                      st, a);
}

}  // namespace pss

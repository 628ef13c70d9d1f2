// pss_persist2d.cuh -- the FP32 2D step as one persistent launch
// (arXiv:2405.02410, section "What cuPSS calculates", Eq. timeupdate).
//
// k2p_step runs n steps of a square FP32 2D field (sides 256, 512, 1024) in
// one cooperative launch of at most one CTA per SM.  Two kinds of field:
// MODE 0, an explicit term M(q) F[(F^-1 m phi)^p] (Models A and B), and
// MODE 1, the KPZ term M(q) F[|grad(F^-1 m h)|^2] (section "Writing models").  Each CTA owns a fixed
// set of half-spectrum columns (pairs kx = 2u, 2u + 1: one Philox call draws
// the noise of both) and a fixed block of rows.  The state phi_q of its
// columns stays in shared memory for the whole launch; only the two work
// arrays of the FFT-group path move through L2 between the phases:
//
//   column phase (step n): P column (x-transformed product) -> forward
//       y-FFT -> update (Eq. timeupdate, noise of step n) -> Hermitian part
//       on kx = 0, Nx/2 -> de-aliased, 1/N_sites-scaled, conjugated kept
//       columns -> y-FFT -> T1 (column-major)
//   grid barrier A
//   row phase: T1 rows of the CTA's row pairs -> C2R along x (two rows as
//       one complex transform) -> power p -> R2C -> P (column-major)
//   grid barrier B
//
// MODE 1 (KPZ): the column phase also transforms i q_y m h back along y (a
// second inverse, array T1a); in the row phase one complex C2R of the two
// rows' i q_x m h and one of their i q_y m h give (d_x h, d_y h) of both rows,
// whose squares, added, are the two rows' products, packed for one R2C.  Three
// transforms per row pair and three per kept column instead of two.
//
// A launch whose product is not in P yet (a fresh state, a new parameter of
// the operators) starts with a prologue: the inverse transforms of the state
// and the row phase, without an update.
//
// The barriers replace the two kernel boundaries of the two-kernel path.
// The transform warps of a CTA meet at named barrier 15; beside them, noise
// warps draw the Philox noise of the CTA's columns one step ahead into two
// shared-memory buffers (the generator has no data dependence, so it fills
// the issue slots the latency-bound transforms leave idle).  A buffer is
// handed over through two mbarriers: "full" (the noise warps have drawn it)
// and "empty" (the update has read it); every wait on them is bounded.  The
// first step's noise is the one the previous launch (or the two-kernel
// path) left drawn ahead in the noise array, and the launch leaves the next
// step's there in turn.  The
// per-mode factors of the update, g = 1 / (1 + dt O(q)) and dt M(q), are
// computed once per launch.
// Every arithmetic operation on the data is the one k2_col / k2_row perform
// (same transforms, same update and noise calls), so the two paths give the
// same bits at the same FFT radix.
//
// The grid barrier is one 64-bit arrival counter in global memory: after a
// CTA barrier of the transform warps, one thread adds 1 with release
// semantics, and all of them poll it with acquire loads until it reaches the
// barrier's target.  The counter is never reset inside a launch; the host
// knows how many arrivals each launch makes and passes the count at the
// launch's start.  Every wait is bounded; a CTA whose wait runs out records
// PSS_STATUS_TIMEOUT, raises the abort word (so that no other CTA waits out
// its own limit) and leaves.  The host clears both words after it has
// reported the error.
#pragma once

#include "pss_fast2d.cuh"

namespace pss {

constexpr int kGridWaitLimit = 1 << 23;   // polls of one grid-barrier wait (about 1 s)

__device__ __forceinline__ unsigned long long ld_acquire_gpu_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned ld_relaxed_gpu(const unsigned *p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_gpu_add(unsigned long long *p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Arrive at a grid barrier: after the CTA's global writes of the phase, the
// NMAIN transform threads meet at named barrier 15 and thread 0 adds the
// CTA's arrival (release: it orders the CTA's writes before it).
template <int NMAIN> __device__ __forceinline__ void grid_arrive(GridSync *gs) {
    asm volatile("bar.sync 15, %0;" ::"n"(NMAIN) : "memory");
    if (threadIdx.x == 0) red_release_gpu_add(&gs->count, 1ull);
}

// Wait until the arrival counter reaches `target` (at most `limit` polls; 0:
// kGridWaitLimit).  Every transform thread calls it; all get the same answer.
// A wait that runs out records the timeout, raises the grid's abort word and
// the CTA's *cta_abort.
template <int NMAIN>
__device__ __forceinline__ bool grid_wait(GridSync *gs, unsigned long long target, int *status, int limit,
                                          volatile int *cta_abort) {
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        int ok = 0;
        if (limit <= 0) limit = kGridWaitLimit;
        // a wait of this CTA that gave up earlier (noise hand-over) ends the launch here,
        // at a point every transform thread reaches
        for (int it = 0; it < limit && !*cta_abort; ++it) {
            if (ld_acquire_gpu_u64(&gs->count) >= target) { ok = 1; break; }
            if ((it & 63) == 63 && (ld_relaxed_gpu(&gs->abort) || *cta_abort)) break;
        }
        if (!ok) {
            if (status) atomicOr(status, kStatusTimeout);
            atomicExch(&gs->abort, 1u);
            *cta_abort = 1;
        }
        s_ok = ok;
    }
    asm volatile("bar.sync 15, %0;" ::"n"(NMAIN) : "memory");
    return s_ok != 0;
}

// CTAs, threads and shared memory of the persistent step.  The transform
// warps are NG = 4 FFT groups of TPF = N / E threads; beside them run NNW
// noise warps.  A CTA owns at most NG / 2 column pairs and NG row pairs.
// Shared memory: mbarriers | roots of unity | state [NG][N] | update factors
// (m, g) [NG][N] (MODE 0) or a third buffer of N points per group (MODE 1) |
// noise, two buffers [2][NG][N] | the groups' buffer pairs.
template <int N, int E, int NNW> struct P2Shape {
    using S = GShape<N, E>;
    static constexpr int NG = 4;
    static constexpr int NMAIN = NG * S::TPF;         // transform threads
    static constexpr int THREADS = NMAIN + 32 * NNW;
    static constexpr size_t BAR = 0;                   // full[2], empty[2]
    static constexpr size_t TW = 128;
    static constexpr size_t ST = TW + sizeof(float2) * N;
    static constexpr size_t MG = ST + sizeof(float2) * NG * N;
    static constexpr size_t NZ = MG + sizeof(float2) * NG * N;
    static constexpr size_t WB = NZ + 2 * sizeof(float2) * NG * N;
    static constexpr size_t BYTES = WB + sizeof(float2) * NG * S::WS;
};

// the CTA's share of `total` units when they are cut into `nb` contiguous blocks
__device__ __forceinline__ void block_range(int total, int nb, int b, int &lo, int &hi) {
    lo = (int)((long long)total * b / nb);
    hi = (int)((long long)total * (b + 1) / nb);
}

// the transform warps' CTA barrier (named barrier 15)
template <int NMAIN> __device__ __forceinline__ void main_sync() {
    asm volatile("bar.sync 15, %0;" ::"n"(NMAIN) : "memory");
}

// mbarrier arrive (release at CTA scope) by the calling thread
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// bounded wait of one thread for phase `parity` of `bar`; gives up early when
// *abort is raised
__device__ __forceinline__ bool mbar_wait_abortable(uint64_t *bar, uint32_t parity, const volatile int *abort) {
    for (int it = 0; it < kWaitLimit; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort) return false;
    }
    return false;
}

// The noise hand-over.  Draw n (the noise of step step0 + n) goes to buffer
// n & 1; draws start at n = first (0 after a prologue, else 1: step 0's
// noise comes from the noise array).  The j-th draw into buffer b completes
// phase j of full[b]; step n's update releases its buffer (empty[b]), and
// draw n >= 2 waits for release number (n - 2 - b) / 2 of its buffer.
__device__ __forceinline__ uint32_t full_parity(int n, int first) {
    const int b = n & 1;
    return (uint32_t)(((n - (b ? 1 : (first ? 2 : 0))) >> 1) & 1);
}
__device__ __forceinline__ uint32_t empty_parity(int n) { return (uint32_t)(((n - 2 - (n & 1)) >> 1) & 1); }

// derivative factor i q of a mode; q = 0 at a Nyquist index, so that the
// derivative of a real field stays real
__device__ __forceinline__ float dq(int k, int n, float g) { return 2 * k == n ? 0.f : fmul(float(signed_k(k, n)), g); }

template <int N, int E, int NNW, int MODE>
__global__ void __launch_bounds__(P2Shape<N, E, NNW>::THREADS, 1) k2p_step(const P2Args a) {
    using C = float2;
    using S = GShape<N, E>;
    using L = P2Shape<N, E, NNW>;
    constexpr int TPF = S::TPF, NG = L::NG, NMAIN = L::NMAIN, H = N / 2 + 1, UC = (H + 1) / 2;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw + L::BAR);     // full[0], full[1]
    uint64_t *empty = full + 2;                                            // empty[0], empty[1]
    C *TW = reinterpret_cast<C *>(smem_raw + L::TW);
    C *ST = reinterpret_cast<C *>(smem_raw + L::ST);   // state of column slot c: ST[c N + ky]
    float2 *MG = reinterpret_cast<float2 *>(smem_raw + L::MG);   // MODE 0: (m, g) of the update per mode
    C *X3 = reinterpret_cast<C *>(smem_raw + L::MG);   // MODE 1: group g's third buffer X3[g N + x]
    C *NZ = reinterpret_cast<C *>(smem_raw + L::NZ);   // noise buffer b of column slot c: NZ[(b NG + c) N + ky]
    C *WB = reinterpret_cast<C *>(smem_raw + L::WB);
    __shared__ FieldP<float> sfp;
    __shared__ unsigned s_step0;
    __shared__ int s_o2;   // offset of the row transforms' results in a group's buffers
    __shared__ volatile int s_abort;   // a wait gave up: every role leaves
    const SysP<float> &sp = a.sp;
    const FieldP<float> &fp = sfp;
    const int t = threadIdx.x;
    const unsigned nb = gridDim.x;
    const int first = a.prologue ? 0 : 1;   // the first noise draw of the launch
    const bool seg = MODE == 0 && a.seg_state != nullptr;   // segment mode
    // this CTA's column pairs [u0, u1) (column slot c = 2 (u - u0) + j holds kx = 2u + j)
    // and row pairs [p0, p1)
    int u0, u1, p0, p1;
    block_range(UC, (int)nb, blockIdx.x, u0, u1);
    block_range(N / 2, (int)nb, blockIdx.x, p0, p1);
    const int ncs = 2 * (u1 - u0);   // column slots in use (the last may lie past Nx/2)
    const int npr = p1 - p0;
    auto kx_of = [&](int c) { return 2 * u0 + c; };

    // ---- set-up (every thread): parameters, step counter, mbarriers
    for (int i = t; i < (int)(sizeof(FieldP<float>) / 4); i += L::THREADS)
        reinterpret_cast<uint32_t *>(&sfp)[i] = reinterpret_cast<const uint32_t *>(a.fps)[i];
    if (t == 0) {
        s_step0 = (unsigned)(*a.d_step);
        // an earlier launch gave up (its barrier words are not yet cleared): leave at once
        s_abort = ld_relaxed_gpu(&a.gs->abort) ? 1 : 0;
        mbar_init(full, 32 * NNW);
        mbar_init(full + 1, 32 * NNW);
        mbar_init(empty, 1);
        mbar_init(empty + 1, 1);
    }
    __syncthreads();   // the only CTA-wide barrier: from here on the two roles run apart
    if (s_abort) return;
    const bool noisy = fp.noisy != 0;

    if (t >= NMAIN) {
        // ================= noise warps =================
        // unit-amplitude noise (times |q|^noise_pow) of steps step0 + first .. step0 + nsteps,
        // one Philox call per (column pair, ky), as noise_range draws it
        const int tn = t - NMAIN;
        const PhiloxKey key = philox_key(fp.seed_lo, fp.seed_hi);
        const int npairs = (u1 - u0) * N;
        for (int n = first; n <= a.nsteps; ++n) {
            const int b = n & 1;
            if (n >= 2 && !mbar_wait_abortable(empty + b, empty_parity(n), &s_abort)) {
                if (!s_abort && a.d_status) atomicOr(a.d_status, kStatusTimeout);
                s_abort = 1;
                return;
            }
            if (noisy) {
                C *nz = NZ + (size_t)b * NG * N;
                const unsigned step = s_step0 + (unsigned)n;
                for (int i = tn; i < npairs; i += 32 * NNW) {
                    const int uu = i >> ilog2(N), ky = i & (N - 1), kx0 = 2 * (u0 + uu);
                    C xa = mk<float>(0.f, 0.f), xb = xa;
                    const float qy = fmul(float(signed_k(ky, N)), sp.gy);
                    const float qx0 = fmul(float(kx0), sp.gx), qx1 = fmul(float(kx0 + 1), sp.gx);
                    const float q2a = q2sum(qx0, qy), q2b = q2sum(qx1, qy);
                    noise_pair<float>(kx0 == 0 || 2 * kx0 == sp.nx, kx0, ky, 0, noise_amp<float>(1.f, fp.noise_pow, q2a),
                                      noise_amp<float>(1.f, fp.noise_pow, q2b), kx0 + 1 < sp.hx, sp,
                                      (uint32_t)fp.field_id, key, step, xa, xb);
                    nz[(2 * uu) * N + ky] = xa;
                    nz[(2 * uu + 1) * N + ky] = xb;
                }
            }
            mbar_arrive(full + b);
        }
        return;
    }

    // ================= transform warps =================
    const int g = t / TPF, gl = t - g * TPF;   // FFT group and its thread
    {
        constexpr int PT = (N + NMAIN - 1) / NMAIN;
        C tv[PT];
#pragma unroll
        for (int q = 0; q < PT; ++q)
            if (t + q * NMAIN < N) tv[q] = __ldg(a.tw + twiddle_offset(N, E) + t + q * NMAIN);
#pragma unroll
        for (int q = 0; q < PT; ++q)
            if (t + q * NMAIN < N) TW[t + q * NMAIN] = tv[q];
    }
    const int kmx = fp.kmax[0], kmy = fp.kmax[1];
    const float scale = sp.inv_nsites;
    const bool has_product = fp.power > 0;
    float dtO[kPolyTerms], dtM[kPolyTerms];
#pragma unroll
    for (int i = 0; i < kPolyTerms; ++i) {
        dtO[i] = sp.dt * fp.O[i];
        dtM[i] = sp.dt * fp.M[i];
    }
    // the state (and, without a prologue, the first step's noise) of each column
    // pair: 16 bytes per (pair, ky) of the tiled arrays (the two columns are
    // neighbours); all of a thread's loads are issued first (their DRAM round trips
    // overlap each other and the update factors below), the stores follow
    constexpr int PERS = 2 * N / NMAIN;   // (pair, ky) items per thread, at most
    const bool load_xi = first == 1 && noisy;
    float4 sv[PERS], xv[PERS];
#pragma unroll
    for (int q = 0; q < PERS; ++q) {
        const int i = t + q * NMAIN, uu = i >> ilog2(N), ky = i & (N - 1), kx0 = 2 * (u0 + uu);
        const size_t o = ((size_t)(kx0 >> 2) * N + ky) * 4 + (kx0 & 3);
        const bool in = i < (u1 - u0) * N;
        sv[q] = in ? __ldcg(reinterpret_cast<const float4 *>(a.state + o)) : make_float4(0.f, 0.f, 0.f, 0.f);
        xv[q] = in && load_xi ? __ldcg(reinterpret_cast<const float4 *>(a.xi + o)) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if constexpr (MODE == 0) {
        for (int c = 0; c < ncs; ++c) {
            const float qx = fmul(float(kx_of(c)), sp.gx);
            for (int ky = t; ky < N; ky += NMAIN) {
                float m, gg;
                update_factors<float>(q2sum(qx, fmul(float(signed_k(ky, N)), sp.gy)), dtO, dtM, m, gg);
                MG[c * N + ky] = make_float2(m, gg);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < PERS; ++q) {
        const int i = t + q * NMAIN, uu = i >> ilog2(N), ky = i & (N - 1), kx0 = 2 * (u0 + uu);
        if (i >= (u1 - u0) * N) break;
        float4 v = sv[q], x = xv[q];
        if (kx0 + 1 >= sp.hx) { v.z = 0.f; v.w = 0.f; x.z = 0.f; x.w = 0.f; }   // past Nx/2
        ST[(2 * uu) * N + ky] = mk<float>(v.x, v.y);
        ST[(2 * uu + 1) * N + ky] = mk<float>(v.z, v.w);
        if (load_xi) {
            NZ[(2 * uu) * N + ky] = mk<float>(x.x, x.y);
            NZ[(2 * uu + 1) * N + ky] = mk<float>(x.z, x.w);
        }
    }
    main_sync<NMAIN>();
    const float sigma0 = fp.sigma0;
    C *gb = WB + g * S::WS;   // this thread's group buffers
    bool alive = true;
    // every transform thread waits for phase `parity` of the noise buffer's
    // "full" mbarrier; the warps agree on the outcome
    auto wait_full = [&](int b, uint32_t parity) {
        if (!mbar_wait_abortable(full + b, parity, &s_abort)) {
            if (!s_abort && a.d_status) atomicOr(a.d_status, kStatusTimeout);
            s_abort = 1;
        }
        main_sync<NMAIN>();
        return !s_abort;
    };
    unsigned long long target = 0;   // the arrival count that ends the next grid barrier

#pragma unroll 1
    for (int n = a.prologue ? -1 : 0; n < a.nsteps && alive; ++n) {
        const bool pro = n < 0;   // the prologue: inverse transforms and row phase of the state, no update
        const int b = n & 1;
        // ================= column phase =================
        // Each FFT group runs its column on its own: the x-transformed product
        // (16-byte asynchronous copies into b1), the forward y-FFT whose last
        // pass applies the update (Eq. timeupdate) mode by mode and writes the
        // de-aliased, scaled, conjugated inverse input into the free buffer, the
        // Hermitian part on the kx = 0, Nx/2 columns, and the y-inverse whose
        // last pass stores T1 (column-major) straight to global memory (MODE 1:
        // then the y-inverse of i q_y times the same input, T1a).
        if (g < ncs) {
            const int kx = kx_of(g);
            C *b0 = gb, *b1 = gb + S::BUF;
            C *U = SinkShape<N, E>::LAST_READS_B1 ? b0 : b1;   // the buffer the last pass does not read
            C *STc = ST + g * N;
            const bool kxk = kx <= kmx, live = kx < sp.hx;
            const bool herm = kx == 0 || kx == N / 2;   // columns whose modes pair up (the field is real)
            C x[E];   // point gl + TPF m of the current transform
            if (!pro) {
                // the x-transformed product of the column straight into the forward
                // transform's first-pass registers
                {
                    const C *Pin = (seg ? a.seg_prod + (size_t)n * a.seg_cstride : a.P) + (size_t)kx * N + gl;
#pragma unroll
                    for (int m = 0; m < E; ++m) x[m] = live ? __ldcg(Pin + m * TPF) : mk<float>(0.f, 0.f);
                }
                // the noise of this step (every thread of the group waits; bounded)
                if (!(n == 0 && first == 1) && !mbar_wait_abortable(full + b, full_parity(n, first), &s_abort)) {
                    if (!s_abort && a.d_status) atomicOr(a.d_status, kStatusTimeout);
                    s_abort = 1;
                }
                const C *nzc = NZ + ((size_t)b * NG + g) * N;
                const float2 *MGc = MG + g * N;
                const float qx = fmul(float(kx), sp.gx);
                // forward y-FFT; its last pass applies the update (Eq. timeupdate) mode by
                // mode and keeps the de-aliased, scaled, conjugated inverse input in x[]
                fft_regs_regs<N, E>(x, b0, b1, gl, 1 + g, TW, [&](int ky, C pq) {
                    const C xi = noisy ? cscale<float>(nzc[ky], sigma0) : mk<float>(0.f, 0.f);
                    float m, gg;
                    if constexpr (MODE == 0) {
                        const float2 mg = MGc[ky];
                        m = mg.x;
                        gg = mg.y;
                    } else {
                        update_factors<float>(q2sum(qx, fmul(float(signed_k(ky, N)), sp.gy)), dtO, dtM, m, gg);
                    }
                    C v = update_pre<float>(STc[ky], pq, xi, m, gg, has_product);
                    if (!live) v = mk<float>(0.f, 0.f);
                    STc[ky] = v;
                    const float sc = (kxk && abs(signed_k(ky, N)) <= kmy) ? scale : 0.f;
                    return mk<float>(v.x * sc, -v.y * sc);
                });
                if (herm) {
                    // Hermitian part: phi(kx, ky) <- (phi(kx, ky) + conj phi(kx, -ky)) / 2, with
                    // the inverse input through shared memory (partner modes sit with other threads)
#pragma unroll
                    for (int m = 0; m < E; ++m) U[gl + m * TPF] = x[m];
                    group_sync<TPF>(1 + g);
                    for (int pos = gl; pos < N / 2 + 1; pos += TPF) {
                        const int ppos = (N - pos) & (N - 1);
                        const C v0 = STc[pos], v1 = STc[ppos];
                        const C h = mk<float>(0.5f * (v0.x + v1.x), 0.5f * (v0.y - v1.y));
                        STc[pos] = h;
                        STc[ppos] = mk<float>(h.x, -h.y);
                        const float s0 = (kxk && abs(signed_k(pos, N)) <= kmy) ? scale : 0.f;
                        const float s1 = (kxk && abs(signed_k(ppos, N)) <= kmy) ? scale : 0.f;
                        U[pos] = mk<float>(h.x * s0, -h.y * s0);
                        U[ppos] = mk<float>(h.x * s1, h.y * s1);
                    }
                    group_sync<TPF>(1 + g);
                }
                if (seg && live) {
                    // the state after step n, tiled, for the adjoint's segment (a thread's own
                    // modes, or any after the Hermitian part's barrier), and the step's unit noise
                    C *so = a.seg_state + (size_t)(n + 1) * a.seg_cstride;
                    C *sz = a.seg_noise && noisy ? a.seg_noise + (size_t)n * a.seg_cstride : nullptr;
#pragma unroll 4
                    for (int m = 0; m < E; ++m) {
                        const int ky = gl + m * TPF;
                        const size_t o = ((size_t)(kx >> 2) * N + ky) * 4 + (kx & 3);
                        so[o] = STc[ky];
                        if (sz) sz[o] = nzc[ky];
                    }
                }
            } else {
                // the inverse input from the state as it is
                for (int ky = gl; ky < N; ky += TPF) {
                    const C v = STc[ky];
                    const float sc = (kxk && abs(signed_k(ky, N)) <= kmy) ? scale : 0.f;
                    U[ky] = mk<float>(v.x * sc, -v.y * sc);
                }
                group_sync<TPF>(1 + g);
            }
            if (kxk) {
                // y-inverse (T1 = F(conj X)), its last pass storing T1 (column-major): from
                // x[] (its first pass into the buffer the forward's last pass did not read),
                // or from U
                C *__restrict__ dst = a.T1 + (size_t)kx * N;
                auto to_t1 = [&](int q, C v) { dst[q] = v; };
                if (!pro && !herm)
                    fft_regs_sink<N, E>(x, U, U == b0 ? b1 : b0, gl, 1 + g, TW, to_t1);
                else
                    fft_fwd_group_sink<N, E>(U == b0 ? b1 : b0, U, gl, 1 + g, TW, to_t1);
                if constexpr (MODE == 1) {
                    // the y-inverse of i q_y X (T1a): its input from the state, into b1
                    group_sync<TPF>(1 + g);
                    for (int ky = gl; ky < N; ky += TPF) {
                        const C v = STc[ky];
                        const float sc = (kxk && abs(signed_k(ky, N)) <= kmy) ? scale : 0.f;
                        const float qd = dq(ky, N, sp.gy);
                        b1[ky] = mk<float>(-qd * v.y * sc, -qd * v.x * sc);   // conj(sc i q_y v)
                    }
                    group_sync<TPF>(1 + g);
                    C *__restrict__ dsta = a.T1a + (size_t)kx * N;
                    fft_fwd_group_sink<N, E>(b0, b1, gl, 1 + g, TW, [&](int q, C v) { dsta[q] = v; });
                }
            }
        }
        // ---- grid barrier A (its CTA barrier also ends the column phase's reads of noise buffer b)
        target += nb;
        if (sp.tx_extra && n == 0 && blockIdx.x == 0) {
            // the bounded-wait check (tuning key "test_timeout"): this CTA never
            // arrives, so the first barrier cannot complete and every wait runs out
            main_sync<NMAIN>();
        } else {
            grid_arrive<NMAIN>(a.gs);
        }
        if (!pro && t == 0) mbar_arrive(empty + b);   // noise buffer b is read: the noise warps may refill it
        alive = grid_wait<NMAIN>(a.gs, target, a.d_status, sp.wait_limit, &s_abort);
        if (!alive) break;
        // ================= row phase =================
        // Each FFT group runs one row pair (rows r0 + 2 g, r0 + 2 g + 1) on its own,
        // from the conjugated y-inverse(s), and the two rows' half spectra of the
        // product go to P (column-major).  The staging of the inputs and the
        // store of the products are shared by the CTA's transform threads: one
        // thread per (column k, row pair j), so that the CTA's rows of a column
        // (2 npr consecutive points of T1 and of P) move as one run.
        if (npr > 0) {
            const int r0 = 2 * p0;   // the CTA's first row
            const int kc = fp.kx_cols;
            C *b0 = gb, *b1 = gb + S::BUF;
            constexpr int PERC = (NG * H + NMAIN - 1) / NMAIN;   // (column, row pair) items per thread
            // stage Y = conj(Z) of every group's rows (as k2_row) into its b1; deriv:
            // times -i q_x first (the conjugate of i q_x)
            auto stage_from = [&](const C *src, bool deriv) {
                float4 v[PERC];
#pragma unroll
                for (int q = 0; q < PERC; ++q) {
                    const int i = t + q * NMAIN, k = i / NG, j = i % NG;
                    v[q] = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (k < kc && j < npr) v[q] = __ldcg(reinterpret_cast<const float4 *>(src + (size_t)k * N + r0 + 2 * j));
                }
#pragma unroll
                for (int q = 0; q < PERC; ++q) {
                    const int i = t + q * NMAIN, k = i / NG, j = i % NG;
                    if (k < H && j < npr) {
                        float ar = v[q].x, ai = v[q].y, br = v[q].z, bi = v[q].w;
                        if (deriv) {
                            const float qd = dq(k, N, sp.gx);
                            const float t0 = qd * ai, t1 = -qd * ar, t2 = qd * bi, t3 = -qd * br;
                            ar = t0; ai = t1; br = t2; bi = t3;
                        }
                        if (k == 0 || k == N / 2) { ai = 0.f; bi = 0.f; }   // the half spectra of real rows
                        const C lo = mk<float>(ar - bi, -ai - br), hi = mk<float>(ar + bi, ai - br);
                        C *bj = WB + j * S::WS + S::BUF;   // group j's b1
                        bj[k] = hi;
                        if (k > 0 && k < N / 2) bj[N - k] = lo;
                    }
                }
                main_sync<NMAIN>();
            };
            // the C2R's last pass hands its outputs to the R2C's first pass in registers
            // (the R2C's first pass writes the buffer that last pass did not read)
            constexpr bool LB1 = SinkShape<N, E>::LAST_READS_B1;
            C *o2 = nullptr;
            if constexpr (MODE == 0) {
                stage_from(a.T1, false);
                if (g < npr) {
                    // segment mode: the de-aliased real rows of the state too
                    float *ra = seg ? a.seg_real + (size_t)(n + 1) * a.seg_rstride + (size_t)(r0 + 2 * g) * N : nullptr;
                    float *rb = ra ? ra + N : nullptr;
                    const int pw = fp.power;
                    C x[E];
                    fft_smem_regs<N, E>(b0, b1, gl, 1 + g, TW, x, [&](int q, C v) {
                        if (ra) {
                            ra[q] = v.x;
                            rb[q] = -v.y;
                        }
                        if (pw > 0) v = mk<float>(pow_p(v.x, pw), pow_p(-v.y, pw));
                        return v;
                    });
                    o2 = fft_regs_smem<N, E>(x, LB1 ? b0 : b1, LB1 ? b1 : b0, gl, 1 + g, TW);
                }
            } else {
                // (d_x h) of both rows as one complex C2R; squares of the two real parts to X3
                C *X = X3 + g * N;
                stage_from(a.T1, true);
                if (g < npr)
                    fft_fwd_group_sink<N, E>(b0, b1, gl, 1 + g, TW,
                                             [&](int q, C v) { X[q] = mk<float>(v.x * v.x, v.y * v.y); });
                main_sync<NMAIN>();
                // (d_y h) of both rows; the sum of squares packs the two rows' products
                stage_from(a.T1a, false);
                if (g < npr) {
                    C x[E];
                    fft_smem_regs<N, E>(b0, b1, gl, 1 + g, TW, x, [&](int q, C v) {
                        return mk<float>(fadd(X[q].x, v.x * v.x), fadd(X[q].y, v.y * v.y));
                    });
                    o2 = fft_regs_smem<N, E>(x, LB1 ? b0 : b1, LB1 ? b1 : b0, gl, 1 + g, TW);
                }
            }
            // every group's result lies at the same offset of its buffers (group 0 always runs)
            if (t == 0) s_o2 = (int)(o2 - gb);
            main_sync<NMAIN>();
            const C *o2w = WB + s_o2;
            C *__restrict__ out = (seg ? a.seg_prod + (size_t)(n + 1) * a.seg_cstride : a.P) + r0;
#pragma unroll
            for (int q = 0; q < PERC; ++q) {
                const int i = t + q * NMAIN, k = i / NG, j = i % NG;
                if (k < H && j < npr) {
                    const C *oj = o2w + j * S::WS;
                    const C wk = oj[k], wm = oj[(N - k) & (N - 1)];
                    *reinterpret_cast<float4 *>(out + (size_t)k * N + 2 * j) =
                        make_float4(0.5f * (wk.x + wm.x), 0.5f * (wk.y - wm.y), 0.5f * (wk.y + wm.y), -0.5f * (wk.x - wm.x));
                }
            }
        }
        // ---- grid barrier B (not after the last step)
        if (n + 1 < a.nsteps) {
            target += nb;
            grid_arrive<NMAIN>(a.gs);
            alive = grid_wait<NMAIN>(a.gs, target, a.d_status, sp.wait_limit, &s_abort);
        }
    }
    if (!alive) {
        s_abort = 1;   // the noise warps stop too
        return;
    }
    // ---- the state, and the next step's unit noise (as the two-kernel path keeps it), back to the
    // tiled arrays; a non-finite mode of the state is reported (it spreads to every mode in a step)
    const int bl = a.nsteps & 1;
    if (!wait_full(bl, full_parity(a.nsteps, first))) return;
    const C *nz = NZ + (size_t)bl * NG * N;
    bool bad = false;
    for (int i = t; i < (seg ? 0 : (u1 - u0) * N); i += NMAIN) {
        const int uu = i >> ilog2(N), ky = i & (N - 1), kx0 = 2 * (u0 + uu);
        const size_t o = ((size_t)(kx0 >> 2) * N + ky) * 4 + (kx0 & 3);
        const C v0 = ST[(2 * uu) * N + ky], v1 = ST[(2 * uu + 1) * N + ky];   // zero past Nx/2
        bad |= !(fabsf(v0.x) + fabsf(v0.y) + fabsf(v1.x) + fabsf(v1.y) <= 3.0e38f);
        *reinterpret_cast<float4 *>(a.state + o) = make_float4(v0.x, v0.y, v1.x, v1.y);
        if (a.xi) {
            const C x0 = noisy ? nz[(2 * uu) * N + ky] : mk<float>(0.f, 0.f);
            const C x1 = noisy ? nz[(2 * uu + 1) * N + ky] : mk<float>(0.f, 0.f);
            *reinterpret_cast<float4 *>(a.xi + o) = make_float4(x0.x, x0.y, x1.x, x1.y);
        }
    }
    if (bad && a.d_status) atomicOr(a.d_status, kStatusNonFinite);
    if (blockIdx.x == 0 && t == 0) *a.d_step = (long long)s_step0 + a.nsteps;
    // the last CTA to finish sets the barrier words back for the next launch
    // (the kernel boundary orders this before that launch's first arrival)
    if (t == 0 && atomicAdd(&a.gs->done, 1u) == nb - 1) {
        a.gs->count = 0ull;
        a.gs->done = 0u;
    }
}

}  // namespace pss

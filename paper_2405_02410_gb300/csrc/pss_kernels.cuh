// pss_kernels.cuh -- the sm_103a kernels of one pseudo-spectral time step
// (arXiv:2405.02410, section "What cuPSS calculates", Eq. timeupdate).
//
// One step of a 2D field runs two kernels; the steady-state schedule is
//   k_col (per kTileW columns, all ky):  forward y-FFT of the x-transformed
//       product -> P_q; Philox noise; semi-implicit update of phi_q (written
//       back); Hermitian part on kx = 0, Nx/2; de-alias mask and 1/N_sites;
//       inverse y-FFT of the kept columns -> T1
//   k_row (per pair of rows):  C2R along x of T1 -> phi^d(x); phi^d(x)^p;
//       R2C along x -> T2 (the next step's product, x-transformed)
// so each step reads and writes phi_q once and moves the product through
// HBM twice.  In 3D the column kernel runs along z, and k_mid adds the y
// passes (inverse before k_row, forward after it).  1D is 2D with one row.
//
// Every kernel stages its input tiles into shared memory with TMA bulk copies
// (one mbarrier, bounded wait), transforms there, does its element-wise work
// in rolled loops over shared memory and writes its outputs with coalesced
// stores.
#pragma once

#include "pss_device.cuh"
#include "pss_internal.h"

namespace pss {

constexpr int W = kTileW;

// Bytes of the roots-of-unity table a kernel with transforms of length N
// stages into shared memory (none below 16 points: one pass, no twiddles).
template <typename C, int N> __host__ __device__ constexpr uint32_t twiddle_bytes() {
    return N >= 16 ? (uint32_t)(N * sizeof(C)) : 0u;
}
// its size in elements (a multiple of 16, so the buffers after it keep their alignment)
template <int N> __host__ __device__ constexpr int twiddle_elems() { return N >= 16 ? N : 0; }

template <typename T> __device__ __forceinline__ T poly5(const T *c, T x) {
    return ffma(ffma(ffma(ffma(c[4], x, c[3]), x, c[2]), x, c[1]), x, c[0]);
}

__device__ __forceinline__ int signed_k(int k, int n) { return k < (n + 1) / 2 ? k : k - n; }

// Noise increments xi_q of two neighbouring modes kx0 = 2j, kx1 = 2j + 1 of
// one row (ky, kz) of the half spectrum (Eq. noise_eq over one step).  Each
// Hermitian pair of modes is drawn once, by its canonical member (the smaller
// index in the half spectrum [kz][ky][kx]); one Philox4x32-10 call, counter
// (((kz Ny + ky) Hxe + kx) / 2, step, field, 0), serves the canonical modes
// 2j and 2j + 1 of a row: words (x0, x1) the even one, (x2, x3) the odd one.
// A mode that is its own partner is real.  amp0/amp1 are the per-component
// standard deviations sqrt(N_sites D~(q) dt / dV) of the two modes.
// on_plane: kx0 is 0 or Nx/2 (its partner is (kx0, -ky, -kz)).
template <typename T>
__device__ __forceinline__ void noise_pair(bool on_plane, int kx0, int ky, int kz, T amp0, T amp1, bool has1,
                                           const SysP<T> &sp, uint32_t fid, const PhiloxKey &key,
                                           uint32_t step, cplx<T> &xi0, cplx<T> &xi1) {
    const uint32_t row = (uint32_t)(kz * sp.ny + ky);
    uint32_t crow = row;
    bool cj = false, selfc = false;
    if (on_plane) {
        const uint32_t prow = (uint32_t)(((sp.nz - kz) & (sp.nz - 1)) * sp.ny + ((sp.ny - ky) & (sp.ny - 1)));
        selfc = prow == row;
        if (prow < row) { crow = prow; cj = true; }
    }
    u32x4 r = philox4x32_10(u32x4{(crow * (uint32_t)sp.hxe + (uint32_t)kx0) >> 1, step, fid, 0u}, key);
    T n1, n2;
    box_muller(uniform24<T>(r.x), uniform24<T>(r.y), n1, n2);
    xi0 = selfc ? mk<T>(T(1.4142135623730951) * amp0 * n1, T(0)) : mk<T>(amp0 * n1, cj ? -amp0 * n2 : amp0 * n2);
    if (has1) {
        // kx1 is odd, so it is never 0 or Nx/2: it is its own canonical member
        if (crow != row)
            r = philox4x32_10(u32x4{(row * (uint32_t)sp.hxe + (uint32_t)kx0) >> 1, step, fid, 0u}, key);
        box_muller(uniform24<T>(r.z), uniform24<T>(r.w), n1, n2);
        xi1 = mk<T>(amp1 * n1, amp1 * n2);
    }
}

// two neighbouring complex values at a 16-byte aligned address (one 16-byte
// access for FP32)
template <typename T> __device__ __forceinline__ void ld_pair(const cplx<T> *p, cplx<T> &a, cplx<T> &b) {
    if constexpr (sizeof(T) == 4) {
        const float4 v = *reinterpret_cast<const float4 *>(p);
        a = mk<T>(v.x, v.y);
        b = mk<T>(v.z, v.w);
    } else {
        a = p[0];
        b = p[1];
    }
}
template <typename T> __device__ __forceinline__ void st_pair(cplx<T> *p, cplx<T> a, cplx<T> b) {
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(a.x, a.y, b.x, b.y);
    } else {
        p[0] = a;
        p[1] = b;
    }
}

// sigma0 |q|^p with |q| = sqrt(q2)
template <typename T> __device__ __forceinline__ T noise_amp(T sigma0, int p, T q2) {
    if (p == 0) return sigma0;
    const T qa = fast_sqrt(q2);
    T amp = sigma0;
    for (int i = 0; i < p; ++i) amp *= qa;
    return amp;
}

// Eq. (timeupdate) with the mode's factors given: g (phi + xi + m P), where
// m = dt M(q) and g = 1 / (1 + dt O(q)) (update_factors)
template <typename T>
__device__ __forceinline__ cplx<T> update_pre(cplx<T> phi, cplx<T> P, cplx<T> xi, T m, T g, bool has_product) {
    T nx = fadd(phi.x, xi.x), ny = fadd(phi.y, xi.y);
    if (has_product) {
        nx = ffma(m, P.x, nx);
        ny = ffma(m, P.y, ny);
    }
    return mk<T>(fmul(nx, g), fmul(ny, g));
}
// the factors m = dt M(q), g = 1 / (1 + dt O(q)) of a mode; dtO, dtM are dt
// times the operator coefficients (O = -L~)
template <typename T> __device__ __forceinline__ void update_factors(T q2, const T *dtO, const T *dtM, T &m, T &g) {
    m = poly5<T>(dtM, q2);
    g = fast_rcp(fadd(T(1), poly5<T>(dtO, q2)));
}
// Eq. (timeupdate): (phi + dt M P + xi) / (1 + dt O)
template <typename T>
__device__ __forceinline__ cplx<T> update_mode(cplx<T> phi, cplx<T> P, cplx<T> xi, T q2, const T *dtO, const T *dtM,
                                               bool has_product) {
    T m, g;
    update_factors<T>(q2, dtO, dtM, m, g);
    return update_pre<T>(phi, P, xi, m, g, has_product);
}

// ---------------------------------------------------------------------------
// k_col: FFTs along the slowest axis (N = n_inner points), fused with the
// update.  A CTA holds F = tiles_per_cta x NP x kTileW columns ("chunks" of
// kTileW columns of one pencil); in 3D the two pencils of a CTA are ky and
// -ky so that the Hermitian partner of every kx = 0 mode sits in the same CTA.
// The CTA has 2 F TPF threads: FFT f = t mod F (consecutive threads,
// consecutive columns), lane t / F; lanes >= TPF only join the element-wise
// phases.  Shared memory: PHI (staged state chunks, [chunk][pos][W] with a
// chunk stride of N W + 8), X (staged product chunks, then a work buffer),
// Y (work buffer).
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// Adjoint of one step, column part (after the forward transform P of the
// kernel's X input along this axis):
//   COL_ADJ_A: PHI = lambda', P = F[r^p] of the step, aux = phi' (global):
//       mu = g lambda' (stored back), gradient sums of the implicit / explicit
//       coefficients and of the noise, and nu = dt M mu transformed back along
//       this axis (all columns, unscaled) -> out.
//   COL_ADJ_B: PHI = mu, P = F[w]: lambda = mu + m F[w] / N (stored back),
//       Hermitian part on the kx = 0, Nx/2 planes.
//   COL_ADJ_BA: the B part of step n, then the A part of step n - 1 on the
//       lambda_n it left in PHI, with P = the forward transform of Z (the
//       product of step n - 1, staged beside X): lambda_n never goes through
//       global memory, and only mu_{n-1} is stored.
// Inner products run over the full Hermitian set: weight 2 for 0 < kx < Nx/2.
// ---------------------------------------------------------------------------
template <typename T, int N, int EMAX>
__device__ __forceinline__ void col_adjoint(const ColArgs<T> &a, const FieldP<T> &fp, cplx<T> *PHI, const cplx<T> *P,
                                            cplx<T> *X, cplx<T> *Y, const cplx<T> *Z, int which, int F, int SF,
                                            int nchunks, int lognch, int first_tile, int op, int opp, int logNP,
                                            size_t sofs, int ch, int c, int f, int lane, bool active,
                                            const cplx<T> *__restrict__ tw) {
    using C = cplx<T>;
    constexpr int CS = N * W + 8;
    const SysP<T> &sp = a.sp;
    const int t = threadIdx.x, nthr = blockDim.x;
    const bool do_b = a.mode != COL_ADJ_A, do_a = a.mode != COL_ADJ_B;
    auto chunk_tile = [&](int q) { return first_tile + (q >> logNP); };
    auto chunk_o = [&](int q) { return (q & logNP) ? opp : op; };
    auto chunk_writes = [&](int q) { return chunk_tile(q) < a.n_tiles && !((q & logNP) && opp == op); };
    auto gofs = [&](int q) { return ((size_t)(chunk_tile(q) * sp.n_outer + chunk_o(q)) * N) * W; };
    const int logF = __ffs(F) - 1;

    if (do_b) {
        // lambda = mu + m F[w] / N on the kept modes
#pragma unroll 1
        for (int i = t; i < N * F; i += nthr) {
            const int pos = i >> logF, ff = i & (F - 1);
            const int chq = ff >> 2, cc = ff & 3;
            const int tile = chunk_tile(chq), kx = tile * W + cc;
            const int o = chunk_o(chq);
            const int ky = sp.dim == 3 ? o : (sp.dim == 2 ? pos : 0);
            const int kz = sp.dim == 3 ? pos : 0;
            const bool valid = tile < a.n_tiles && kx < sp.hx;
            const bool keep = valid && kx <= fp.kmax[0] && abs(signed_k(ky, sp.ny)) <= fp.kmax[1] &&
                              abs(signed_k(kz, sp.nz)) <= fp.kmax[2];
            C *ph = &PHI[chq * CS + pos * W + cc];
            const C pv = P[ff * SF + spad(pos)];
            const C mu = *ph;
            *ph = keep ? mk<T>(mu.x + pv.x * sp.inv_nsites, mu.y + pv.y * sp.inv_nsites) : (valid ? mu : mk<T>(0, 0));
        }
        __syncthreads();
        // Hermitian part of lambda on the kx = 0, Nx/2 planes
        const int last_tile = first_tile + a.tiles_per_cta;
        if (first_tile == 0 || (first_tile * W <= sp.nx / 2 && sp.nx / 2 < last_tile * W)) {
#pragma unroll 1
            for (int i = t; i < N * F; i += nthr) {
                const int pos = i >> logF, ff = i & (F - 1);
                const int cq = ff >> 2, cc = ff & 3;
                const int kq = chunk_tile(cq) * W + cc;
                if (!(kq == 0 || 2 * kq == sp.nx) || (cq & logNP) != 0) continue;
                const int ppos = (N - pos) & (N - 1);
                if (logNP == 0 && ppos < pos) continue;
                C *p0 = &PHI[cq * CS + pos * W + cc];
                C *p1 = &PHI[(cq + logNP) * CS + ppos * W + cc];
                const C u0 = *p0, u1 = *p1;
                const C h = mk<T>(T(0.5) * (u0.x + u1.x), T(0.5) * (u0.y - u1.y));
                *p0 = h;
                *p1 = mk<T>(h.x, -h.y);
            }
            __syncthreads();
        }
        if (a.mode == COL_ADJ_BA) {
            // the A part's P: forward transform of the earlier step's product
            const int zstride = a.in2_colmajor ? 1 : W;
            const C *zb = Z + ch * CS + (a.in2_colmajor ? c * N : c);
            which = fft_run<T, N, EMAX, -1>([&](int p) { return zb[p * zstride]; },
                                            [&](int p, C v, C *fr) { fr[spad(p)] = v; },
                                            Y + f * SF, X + f * SF, lane, active, tw);
            __syncthreads();
            P = which == 0 ? Y : X;
        }
    }

    // A part: nu goes into the work buffer that does not hold P
    C *NU = which == 0 ? X : Y;
    // a thread's partial sums over its few modes are in the working precision;
    // the sums over threads, CTAs and time steps are FP64
    using Acc = T;
    Acc acc[11];
#pragma unroll
    for (int i = 0; i < 11; ++i) acc[i] = Acc(0);
    if (do_a) {
        const uint32_t step = (uint32_t)(a.adj_step + (a.d_adj_base ? *a.d_adj_base : 0));
        const PhiloxKey key = philox_key(fp.seed_lo, fp.seed_hi);
        // one iteration per pair of neighbouring columns at one position: a single
        // Philox draw serves both modes of the pair
#pragma unroll 1
        for (int j = t; j < (N * F) >> 1; j += nthr) {
            const int pos = j >> (logF - 1), ff0 = (j & ((F >> 1) - 1)) << 1;
            const int chq = ff0 >> 2, cc0 = ff0 & 3;
            const int tile = chunk_tile(chq);
            const int kx0 = tile * W + cc0;
            const int o = chunk_o(chq);
            const int ky = sp.dim == 3 ? o : (sp.dim == 2 ? pos : 0);
            const int kz = sp.dim == 3 ? pos : 0;
            const T qy = T(signed_k(ky, sp.ny)) * sp.gy, qz = T(signed_k(kz, sp.nz)) * sp.gz;
            C xin[2] = {mk<T>(0, 0), mk<T>(0, 0)};
            if (fp.noisy && tile < a.n_tiles && kx0 < sp.hx && chunk_writes(chq)) {
                const T qe = T(kx0) * sp.gx, qo = T(kx0 + 1) * sp.gx;
                const T q2e = qe * qe + qy * qy + qz * qz, q2o = qo * qo + qy * qy + qz * qz;
                noise_pair<T>(kx0 == 0 || 2 * kx0 == sp.nx, kx0, ky, kz, noise_amp<T>(fp.sigma0, fp.noise_pow, q2e),
                              noise_amp<T>(fp.sigma0, fp.noise_pow, q2o), kx0 + 1 < sp.hx, sp, (uint32_t)fp.field_id,
                              key, step, xin[0], xin[1]);
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int ff = ff0 + u, cc = cc0 + u, kx = kx0 + u;
                const bool valid = tile < a.n_tiles && kx < sp.hx;
                const T qx = T(kx) * sp.gx;
                const T q2 = qx * qx + qy * qy + qz * qz;
                C *ph = &PHI[chq * CS + pos * W + cc];
                const C pv = P[ff * SF + spad(pos)];
                const T g = T(1) / (T(1) + sp.dt * poly5<T>(fp.O, q2));
                const C mu = valid ? cscale<T>(*ph, g) : mk<T>(0, 0);
                *ph = mu;
                const T dtM = fp.power > 0 ? sp.dt * poly5<T>(fp.M, q2) : T(0);
                NU[ff * SF + spad(pos)] = cscale<T>(mu, dtM);
                // the duplicate pencil of a self-paired 3D CTA does not count twice
                if (valid && chunk_writes(chq)) {
                    const Acc wgt = (kx == 0 || 2 * kx == sp.nx) ? Acc(1) : Acc(2);
                    const C phin = a.aux[sofs + gofs(chq) + pos * W + cc];
                    const Acc a_phi = wgt * sp.dt * (mu.x * phin.x + mu.y * phin.y);
                    const Acc a_P = wgt * sp.dt * (mu.x * pv.x + mu.y * pv.y);
                    Acc q2k = Acc(1);
#pragma unroll
                    for (int k = 0; k < 5; ++k) {
                        acc[k] -= q2k * a_phi;
                        acc[5 + k] += q2k * a_P;
                        q2k *= q2;
                    }
                    if (fp.noisy) acc[10] += wgt * (mu.x * xin[u].x + mu.y * xin[u].y);
                }
            }
        }
        __syncthreads();
        // CTA reduction of the gradient sums, one FP64 atomic per value.  In
        // FP32 the warp sum is compensated (TwoSum: hi + lo holds it to about
        // the square of FP32 rounding) and only its result goes to FP64, once
        // per warp: FP64 arithmetic runs at a small fraction of the FP32 rate
        // on this GPU, and a butterfly of FP64 adds on every lane cost more
        // than the rest of the update
        __shared__ double red[11];
        if (t < 11) red[t] = 0.0;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 11; ++k) {
            double v;
            if constexpr (std::is_same<Acc, float>::value) {
                float hi = acc[k], lo = 0.f;
                for (int o = 16; o > 0; o >>= 1) {
                    const float ohi = __shfl_xor_sync(0xffffffffu, hi, o);
                    const float olo = __shfl_xor_sync(0xffffffffu, lo, o);
                    const float s = __fadd_rn(hi, ohi), bp = __fsub_rn(s, hi);
                    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(ohi, bp));
                    hi = s;
                    lo = __fadd_rn(__fadd_rn(lo, olo), err);
                }
                if ((t & 31) == 0) {
                    v = (double)hi + (double)lo;
                    if (v != 0.0) atomicAdd(&red[k], v);
                }
            } else {
                v = (double)acc[k];
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if ((t & 31) == 0 && v != 0.0) atomicAdd(&red[k], v);
            }
        }
        __syncthreads();
        if (t < 11 && red[t] != 0.0) atomicAdd(&a.grad[(size_t)(a.slot0 + blockIdx.z) * 11 + t], red[t]);
    }
    // store PHI (mu or lambda) back with one bulk copy per chunk
    fence_proxy_async();
    __syncthreads();
    const uint32_t chunk_bytes = (uint32_t)(N * W * sizeof(C));
    if (t == 0) {
        for (int q = 0; q < nchunks; ++q)
            if (chunk_writes(q)) bulk_s2g(a.state + sofs + gofs(q), PHI + q * CS, chunk_bytes);
        bulk_commit();
    }
    if (do_a) {
        // nu back along this axis (all columns), stored straight from the last pass
        C *__restrict__ dst = a.out + sofs + gofs(ch) + c;
        const bool writes = chunk_writes(ch);
        C *nb = NU + f * SF;
        C *other = (NU == X ? Y : X) + f * SF;
        fft_run<T, N, EMAX, +1>([&](int p) { return nb[spad(p)]; },
                          [&](int p, C v, C *) {
                              if (writes) dst[p * W] = v;
                          },
                          other, nb, lane, active, tw);
    }
    if (t == 0) bulk_wait_read();
}

template <typename T, int N> struct ColSmem {
    static constexpr int CS = N * W + 8;                         // chunk stride (elements)
    __host__ __device__ static int xs(int F) {                   // X / Y size (elements)
        const int a = F * sf_fft_fastest(N, F), b = (F / W) * CS;
        return a > b ? a : b;
    }
    __host__ __device__ static size_t bytes(int F) {
        return 128 + sizeof(cplx<T>) * ((size_t)twiddle_elems<N>() + (size_t)(F / W) * CS + 2 * (size_t)xs(F));
    }
    // the adjoint instantiation also stages COL_ADJ_BA's second product (Z, after Y)
    __host__ __device__ static size_t bytes_adj(int F) { return bytes(F) + sizeof(cplx<T>) * (size_t)(F / W) * CS; }
};

template <typename T, int N, int EMAX, bool ADJ>
__global__ void __launch_bounds__(512, (N >= 512 || ADJ) ? 1 : 2) k_col(const ColArgs<T> a) {
    using C = cplx<T>;
    using L = ColSmem<T, N>;
    constexpr int TPF = FftShape<N, EMAX>::TPF;
    constexpr int CS = L::CS;
    constexpr int LOGNW = FftShape<N, EMAX>::LOG + 2;                 // log2(N W)
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);
    const int F = a.F;                                           // a power of two, multiple of W
    const int logF = __ffs(F) - 1;
    const int nchunks = F / W, lognch = logF - 2;
    const int SF = sf_fft_fastest(N, F);
    C *TW = reinterpret_cast<C *>(smem_raw + 128);             // roots of unity of length N
    C *PHI = TW + twiddle_elems<N>();
    C *X = PHI + nchunks * CS;
    C *Y = X + L::xs(F);
    C *Z = Y + L::xs(F);                                          // COL_ADJ_BA only
    const SysP<T> &sp = a.sp;
    const int slot = a.slot0 + blockIdx.z;
    // the slot's parameters and the step number, fetched into shared memory
    // while the bulk copies are in flight
    __shared__ FieldP<T> sfp;
    __shared__ uint32_t sstep;
    const FieldP<T> &fp = sfp;
    const size_t sofs = (size_t)slot * a.slot_stride;
    const int logNP = sp.dim == 3 ? 1 : 0;
    const int t = threadIdx.x, nthr = blockDim.x;
    const int op = blockIdx.y;
    const int opp = (sp.n_outer - op) & (sp.n_outer - 1);        // partner pencil (-ky)
    const int mode = a.mode;
    const int first_tile = blockIdx.x * a.tiles_per_cta;
    const C *__restrict__ tw = TW;

    auto chunk_tile = [&](int ch) { return first_tile + (ch >> logNP); };
    auto chunk_o = [&](int ch) { return (ch & logNP) ? opp : op; };
    auto chunk_ok = [&](int ch) { return chunk_tile(ch) < a.n_tiles; };
    auto chunk_writes = [&](int ch) { return chunk_ok(ch) && !((ch & logNP) && opp == op); };
    auto gofs = [&](int ch) { return ((size_t)(chunk_tile(ch) * sp.n_outer + chunk_o(ch)) * N) * W; };

    // ---- stage: state chunks -> PHI (not for COL_FWD), product chunks -> X (COL_STEP, COL_FWD)
    constexpr bool adj = ADJ;   // the adjoint modes are a separate instantiation
    const bool need_in = mode == COL_STEP || mode == COL_FWD || adj;
    const bool need_phi = mode != COL_FWD;
    const bool need_in2 = adj && mode == COL_ADJ_BA;
    const uint32_t chunk_bytes = (uint32_t)(N * W * sizeof(C));
    int nvalid = 0;                                              // chunks 0..nvalid-1 lie inside the grid
    for (int ch = 0; ch < nchunks; ++ch) nvalid += chunk_ok(ch) ? 1 : 0;
    pdl_wait();
    pdl_trigger();
    if (t == 0) {
        mbar_init(bar, 1);
        // (tx_extra: the bounded-wait check makes the first CTA expect more
        // bytes than its copies deliver, so that its wait runs out)
        const uint32_t extra = (blockIdx.x | blockIdx.y | blockIdx.z) == 0 ? sp.tx_extra : 0u;
        mbar_expect_tx(bar, chunk_bytes * nvalid * ((need_in ? 1 : 0) + (need_phi ? 1 : 0) + (need_in2 ? 1 : 0)) +
                                twiddle_bytes<C, N>() + extra);
        if (twiddle_bytes<C, N>()) bulk_g2s(TW, a.tw + twiddle_offset(N, EMAX), twiddle_bytes<C, N>(), bar);
        for (int ch = 0; ch < nvalid; ++ch) {
            if (need_phi) bulk_g2s(PHI + ch * CS, a.state + sofs + gofs(ch), chunk_bytes, bar);
            if (need_in) bulk_g2s(X + ch * CS, a.in + sofs + gofs(ch), chunk_bytes, bar);
            if (need_in2) bulk_g2s(Z + ch * CS, a.in2 + sofs + gofs(ch), chunk_bytes, bar);
        }
    }
    static_assert(sizeof(FieldP<T>) % 4 == 0, "FieldP is copied as 32-bit words");
    for (int i = t; i < (int)(sizeof(FieldP<T>) / 4); i += (int)blockDim.x)   // CTAs may be smaller than FieldP
        reinterpret_cast<uint32_t *>(&sfp)[i] = reinterpret_cast<const uint32_t *>(&a.fps[slot])[i];
    if (t == 0) sstep = (uint32_t)(*a.d_step);
    __syncthreads();   // the barrier is initialised before anyone polls it
    for (int i = nvalid * (N * W) + t; i < nchunks * (N * W); i += nthr) {   // chunks past the last tile read as zero
        const int ch = i >> LOGNW, r = i & (N * W - 1);
        PHI[ch * CS + r] = mk<T>(0, 0);
        X[ch * CS + r] = mk<T>(0, 0);
        if (need_in2) Z[ch * CS + r] = mk<T>(0, 0);
    }
    if (!mbar_wait_all(bar, 0, a.d_status, sp.wait_limit)) return;

    // this thread's FFT: column c of chunk ch
    const int f = t & (F - 1), lane = t >> logF;
    const bool active = lane < TPF;
    const int ch = f >> 2, c = f & 3;
    const int my_tile = chunk_tile(ch), my_o = chunk_o(ch);
    const int kx = my_tile * W + c;

    if (need_in) {
        // forward transform along this axis: P_q (the staged chunk is [pos][W],
        // or [W][pos] for a column-major input)
        const int xstride = a.in_colmajor ? 1 : W;
        const C *xb = X + ch * CS + (a.in_colmajor ? c * N : c);
        int which = 0;
        if (!ADJ && mode == COL_STEP && fp.spectral) {
            // the product arrives transformed along every axis (several product
            // terms with different operators, summed in Fourier space): only
            // its layout changes
#pragma unroll 1
            for (int i = t; i < N * F; i += nthr) {
                const int ff = i & (F - 1), pos = i >> logF;
                Y[ff * SF + spad(pos)] = X[(ff >> 2) * CS + pos * W + (ff & 3)];
            }
        } else {
            which = fft_run<T, N, EMAX, -1>([&](int p) { return xb[p * xstride]; },
                                            [&](int p, C v, C *fr) { fr[spad(p)] = v; },
                                            Y + f * SF, X + f * SF, lane, active, tw);
        }
        __syncthreads();
        const C *P = which == 0 ? Y : X;
        if constexpr (ADJ) {
            col_adjoint<T, N, EMAX>(a, fp, PHI, P, X, Y, Z, which, F, SF, nchunks, lognch, first_tile, op, opp, logNP,
                                    sofs, ch, c, f, lane, active, tw);
            return;
        }
        const uint32_t step = sstep;
        // update: each thread keeps one pair of neighbouring columns (they share
        // one Philox draw) of one chunk and walks the positions
        const int cp = t & 1, chq = (t >> 1) & (nchunks - 1);
        const int pos_step = nthr >> (1 + lognch);
        const int tile = chunk_tile(chq), o = chunk_o(chq);
        const int c0 = 2 * cp, kx0 = tile * W + c0;
        const bool has0 = kx0 < sp.hx, has1 = kx0 + 1 < sp.hx;
        const bool on_plane = kx0 == 0 || 2 * kx0 == sp.nx;
        const T qx0 = T(kx0) * sp.gx, qx1 = T(kx0 + 1) * sp.gx;
        const T qx0s = qx0 * qx0, qx1s = qx1 * qx1;
        const C *P0 = P + (chq * W + c0) * SF, *P1 = P0 + SF;
        C *phb = PHI + chq * CS + c0;
        bool bad = false;
        T dtO[kPolyTerms], dtM[kPolyTerms];
#pragma unroll
        for (int i = 0; i < kPolyTerms; ++i) {
            dtO[i] = sp.dt * fp.O[i];
            dtM[i] = sp.dt * fp.M[i];
        }
        const bool has_product = fp.power > 0, noisy = fp.noisy != 0;
        const int noise_pow = fp.noise_pow, fid = fp.field_id;
        const T sigma0 = fp.sigma0;
        const PhiloxKey key = philox_key(fp.seed_lo, fp.seed_hi);
        if (tile < a.n_tiles) {
#pragma unroll 1
            for (int pos = t >> (1 + lognch); pos < N; pos += pos_step) {
                C v0 = P0[spad(pos)], v1 = P1[spad(pos)];
                C *ph = phb + pos * W;
                if (mode == COL_STEP) {
                    C f0, f1;
                    ld_pair<T>(ph, f0, f1);
                    const int ky = sp.dim == 3 ? o : (sp.dim == 2 ? pos : 0);
                    const int kz = sp.dim == 3 ? pos : 0;
                    const T qy = T(signed_k(ky, sp.ny)) * sp.gy, qz = T(signed_k(kz, sp.nz)) * sp.gz;
                    const T qyz2 = qy * qy + qz * qz;
                    const T q2a = qx0s + qyz2, q2b = qx1s + qyz2;
                    C xi0 = mk<T>(0, 0), xi1 = mk<T>(0, 0);
                    if (noisy)
                        noise_pair<T>(on_plane, kx0, ky, kz, noise_amp<T>(sigma0, noise_pow, q2a),
                                      noise_amp<T>(sigma0, noise_pow, q2b), has1, sp, (uint32_t)fid, key,
                                      step, xi0, xi1);
                    v0 = update_mode<T>(f0, v0, xi0, q2a, dtO, dtM, has_product);
                    v1 = update_mode<T>(f1, v1, xi1, q2b, dtO, dtM, has_product);
                    // false for NaN and for infinities (or values next to overflow)
                    bad |= !(fabs(v0.x) + fabs(v0.y) + fabs(v1.x) + fabs(v1.y) <= T(sizeof(T) == 4 ? 3.0e38 : 1.0e300));
                }
                st_pair<T>(ph, has0 ? v0 : mk<T>(0, 0), has1 ? v1 : mk<T>(0, 0));
            }
        }
        if (bad && a.d_status) atomicOr(a.d_status, kStatusNonFinite);
        __syncthreads();
        // Hermitian part on the kx = 0 and kx = Nx/2 planes (the field is real):
        // phi(kx, k) <- (phi(kx, k) + conj phi(kx, -k)) / 2, each pair by one thread.
        // The CTA holds at most these two plane columns (chunk of the first
        // pencil, column within the chunk); the partner of position pos sits at
        // -pos of the same chunk (2D) or of the partner pencil's chunk (3D).
        int pl_cq0 = 0, pl_cc0 = 0, pl_cq1 = 0, pl_cc1 = 0, npl = 0;
        if (first_tile == 0) ++npl;
        {
            const int kh = sp.nx / 2, last_tile = first_tile + a.tiles_per_cta;
            if (kh > 0 && first_tile * W <= kh && kh < last_tile * W) {
                const int cqh = (kh / W - first_tile) << logNP, cch = kh & (W - 1);
                if (npl == 0) { pl_cq0 = cqh; pl_cc0 = cch; } else { pl_cq1 = cqh; pl_cc1 = cch; }
                ++npl;
            }
        }
        if (npl > 0) {
            constexpr int LOGN = FftShape<N, EMAX>::LOG;
#pragma unroll 1
            for (int i = t; i < (npl << LOGN); i += nthr) {
                const int j = i >> LOGN, pos = i & (N - 1);
                const int cq = j ? pl_cq1 : pl_cq0, cc = j ? pl_cc1 : pl_cc0;
                const int ppos = (N - pos) & (N - 1);
                if (logNP == 0 && ppos < pos) continue;
                C *p0 = &PHI[cq * CS + pos * W + cc];
                C *p1 = &PHI[(cq + logNP) * CS + ppos * W + cc];
                const C u0 = *p0, u1 = *p1;
                const C h = mk<T>(T(0.5) * (u0.x + u1.x), T(0.5) * (u0.y - u1.y));
                *p0 = h;
                *p1 = mk<T>(h.x, -h.y);
            }
            __syncthreads();
        }
        // write the state back: one bulk copy per chunk (contiguous in global memory)
        fence_proxy_async();   // every thread's PHI writes, before the copy engine reads them
        __syncthreads();
        if (t == 0) {
            cplx<T> *sdst = a.state_out ? a.state_out : a.state;
            for (int cq = 0; cq < nvalid; ++cq)
                if (chunk_writes(cq)) bulk_s2g(sdst + sofs + gofs(cq), PHI + cq * CS, chunk_bytes);
            bulk_commit();
        }
        if (mode == COL_FWD) {
            if (t == 0) bulk_wait_read();
            return;
        }
    }

    // ---- inverse along this axis of the de-aliased (not for COL_INV_FULL),
    // 1/N_sites-scaled field, stored straight from the last pass
    const bool full = mode == COL_INV_FULL;
    bool skip = false;
    if (!full) {
        const bool ky_kept = sp.dim != 3 || abs(signed_k(op, sp.ny)) <= fp.kmax[1];
        skip = first_tile * W > fp.kmax[0] || !ky_kept;              // CTA-uniform: nothing kept
    }
    if (!skip) {
        __syncthreads();   // PHI is final; X and Y are free
        const bool kx_keep = kx < sp.hx && (full || kx <= fp.kmax[0]);
        const bool o_keep = full || sp.dim != 3 || abs(signed_k(my_o, sp.ny)) <= fp.kmax[1];
        const int kmax_pos = full ? N : (sp.dim == 3 ? fp.kmax[2] : (sp.dim == 2 ? fp.kmax[1] : 0));
        const T scale = (kx_keep && o_keep) ? sp.inv_nsites : T(0);
        const C *pb = PHI + ch * CS + c;
        const bool writes = chunk_writes(ch) && (full || my_tile * W <= fp.kmax[0]);
        C *__restrict__ dst = a.out + sofs + gofs(ch) + c;
        // a product-term factor: op(q) = (i q_d) (-q^2)^l, q_d = 0 at a Nyquist index
        const T gpos = sp.dim == 3 ? sp.gz : sp.gy;
        const T qx = T(kx) * sp.gx, qo = sp.dim == 3 ? T(signed_k(my_o, sp.ny)) * sp.gy : T(0);
        const int dpos = sp.dim == 3 ? 2 : 1;                    // the axis of this kernel's transform
        auto op = [&](int p, C v) {
            const T qp = T(signed_k(p, N)) * gpos;
            const T qy = sp.dim == 3 ? qo : qp, qz = sp.dim == 3 ? qp : T(0);
            T f = T(1);
            for (int l = 0; l < a.op_lap; ++l) f *= -(qx * qx + qy * qy + qz * qz);
            if (a.op_deriv < 0) return cscale<T>(v, f);
            T q;
            if (a.op_deriv == 0) q = 2 * kx == sp.nx ? T(0) : qx;
            else if (a.op_deriv == dpos) q = 2 * p == N ? T(0) : qp;
            else q = 2 * my_o == sp.ny ? T(0) : qo;              // y in 3D
            return mk<T>(-q * f * v.y, q * f * v.x);
        };
        auto sink = [&](int p, C v, C *) {
            if (writes) dst[p * W] = v;
        };
        // two call sites, so that the step's inverse carries no per-element test
        if (a.op_on)
            fft_run<T, N, EMAX, +1>(
                [&](int p) {
                    return abs(signed_k(p, N)) <= kmax_pos ? op(p, cscale<T>(pb[p * W], scale)) : mk<T>(0, 0);
                },
                sink, X + f * SF, Y + f * SF, lane, active, tw);
        else
            fft_run<T, N, EMAX, +1>(
                [&](int p) { return abs(signed_k(p, N)) <= kmax_pos ? cscale<T>(pb[p * W], scale) : mk<T>(0, 0); },
                sink, X + f * SF, Y + f * SF, lane, active, tw);
    }
    if (need_in && t == 0) bulk_wait_read();   // PHI must outlive the state write-back
}

// ---------------------------------------------------------------------------
// k_row: transforms along x (N = nx) for G pairs of rows per CTA.  Two real
// rows a, b ride on one complex FFT z = a + i b: C2R builds
// Z_k = A_k + i B_k from the two half spectra, and R2C splits the transform W
// of z by A_k = (W_k + conj W_{N-k}) / 2, B_k = (W_k - conj W_{N-k}) / (2i).
// Threads: lane t mod TPF of pair t / TPF.  Shared memory: S (the staged
// input, tile segments of 2G rows with a stride of 2G W + 4; also a work
// buffer), B0, B1 (work buffers).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ size_t real_row_offset(const SysP<T> &sp, int row) {
    if (sp.dim == 3) {
        const int y = row / sp.nz, z = row % sp.nz;
        return ((size_t)z * sp.ny + y) * sp.nx;
    }
    return (size_t)row * sp.nx;
}

template <typename T> __device__ __forceinline__ T ipow(T x, int p) {
    T r = T(1);
    for (int i = 0; i < p; ++i) r *= x;
    return r;
}

template <typename T, int N> struct RowSmem {
    __host__ __device__ static int tstride(int G) { return 2 * G * W + 4; }
    __host__ __device__ static int s_elems(int G, int ntiles) {
        int a = ntiles * tstride(G), b = G * N, c = G * sf_row(N);   // tiles, 2G real rows, work
        a = a > b ? a : b;
        return a > c ? a : c;
    }
    __host__ __device__ static size_t bytes(int G, int ntiles) {
        return 128 + sizeof(cplx<T>) * ((size_t)twiddle_elems<N>() + (size_t)s_elems(G, ntiles) + 2 * (size_t)G * sf_row(N));
    }
};

template <typename T, int N, int EMAX>
__global__ void __launch_bounds__(256) k_row(const RowArgs<T> a) {
    using C = cplx<T>;
    using L = RowSmem<T, N>;
    constexpr int TPF = FftShape<N, EMAX>::TPF;
    constexpr int SF = sf_row(N);
    constexpr int LOGTPF = FftShape<N, EMAX>::LOG - FftShape<N, EMAX>::LOGE;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);
    const SysP<T> &sp = a.sp;
    const int G = a.G, G2 = 2 * a.G;                            // G a power of two
    const int logG = __ffs(G) - 1;
    const int TS = L::tstride(G);
    C *TW = reinterpret_cast<C *>(smem_raw + 128);             // roots of unity of length N
    C *S = TW + twiddle_elems<N>();
    T *Sr = reinterpret_cast<T *>(S);
    C *B0 = S + L::s_elems(G, sp.ntiles);
    C *B1 = B0 + G * SF;
    const int slot = a.slot0 + blockIdx.y;
    __shared__ FieldP<T> sfp;                                  // the slot's parameters, fetched during the copies
    const FieldP<T> &fp = sfp;
    const size_t sofs = (size_t)slot * a.slot_stride;
    const int t = threadIdx.x, nthr = blockDim.x;
    const int r0 = blockIdx.x * G2;
    const int rows = sp.rows;
    const int nrow = rows - r0 < G2 ? rows - r0 : G2;          // rows present in this CTA
    const int mode = a.mode;
    const C *__restrict__ tw = TW;
    pdl_wait();
    pdl_trigger();

    // ---- stage the input rows
    if (mode == ROW_R2C) {
        const T *__restrict__ src = a.real_in + (size_t)slot * a.real_stride;
        const uint32_t row_bytes = (uint32_t)(N * sizeof(T));
        if (t == 0) {
            mbar_init(bar, 1);
            mbar_expect_tx(bar, row_bytes * nrow + twiddle_bytes<C, N>());
            if (twiddle_bytes<C, N>()) bulk_g2s(TW, a.tw + twiddle_offset(N, EMAX), twiddle_bytes<C, N>(), bar);
            for (int rl = 0; rl < nrow; ++rl) bulk_g2s(Sr + rl * N, src + real_row_offset(sp, r0 + rl), row_bytes, bar);
        }
        __syncthreads();   // the barrier is initialised before anyone polls it
        for (int i = nrow * N + t; i < G2 * N; i += nthr) Sr[i] = T(0);
    } else {
        const C *__restrict__ src = a.in + sofs;
        const int kxc_in = (mode == ROW_FUSED || mode == ROW_C2R_KEPT) ? a.kx_cols_max : sp.hx;
        const int ntl = (kxc_in + W - 1) / W;
        const uint32_t seg = (uint32_t)(nrow * W * sizeof(C));
        if (t == 0) {
            mbar_init(bar, 1);
            mbar_expect_tx(bar, seg * ntl + twiddle_bytes<C, N>());
            if (twiddle_bytes<C, N>()) bulk_g2s(TW, a.tw + twiddle_offset(N, EMAX), twiddle_bytes<C, N>(), bar);
        }
        __syncthreads();
        for (int tl = t; tl < ntl; tl += nthr) bulk_g2s(S + tl * TS, src + ((size_t)tl * rows + r0) * W, seg, bar);
        if (nrow < G2)
            for (int i = t; i < ntl * G2 * W; i += nthr) {
                const int tl = i / (G2 * W), r = i - tl * (G2 * W);
                if (r / W >= nrow) S[tl * TS + r] = mk<T>(0, 0);
            }
    }
    static_assert(sizeof(FieldP<T>) % 4 == 0, "FieldP is copied as 32-bit words");
    for (int i = t; i < (int)(sizeof(FieldP<T>) / 4); i += nthr)
        reinterpret_cast<uint32_t *>(&sfp)[i] = reinterpret_cast<const uint32_t *>(&a.fps[slot])[i];
    if (!mbar_wait_all(bar, 0, a.d_status)) return;

    const int lane = t & (TPF - 1), g = t >> LOGTPF;
    const bool active = g < G;
    C *b0 = B0 + g * SF, *b1 = B1 + g * SF;
    auto smem_sink = [&](int p, C v, C *fr) { fr[spad(p)] = v; };
    const C *R;          // this CTA's result buffer (B0 or B1)
    if (mode == ROW_R2C) {
        const int which = fft_run<T, N, EMAX, -1>([&](int p) { return mk<T>(Sr[g * N + p], Sr[(G + g) * N + p]); },
                                            smem_sink, b0, b1, lane, active, tw);
        R = which == 0 ? B0 : B1;
    } else {
        const int kxc = (mode == ROW_FUSED || mode == ROW_C2R_KEPT) ? fp.kx_cols : sp.hx;
        const int which = fft_run<T, N, EMAX, +1>(
            [&](int k) {
                const int kk = k <= N / 2 ? k : N - k;
                C xa = mk<T>(0, 0), xb = mk<T>(0, 0);
                if (kk < kxc) {
                    const int base = (kk >> 2) * TS + (kk & 3);
                    xa = S[base + g * W];
                    xb = S[base + (G + g) * W];
                }
                if (k > N / 2) { xa.y = -xa.y; xb.y = -xb.y; }
                if (k == 0 || 2 * k == N) { xa.y = T(0); xb.y = T(0); }
                return mk<T>(xa.x - xb.y, xa.y + xb.x);
            },
            smem_sink, b0, b1, lane, active, tw);
        __syncthreads();
        C *Z = which == 0 ? B0 : B1;
        if (mode == ROW_C2R || mode == ROW_C2R_KEPT) {
            if (a.fac_acc) {
                // a product-term factor: r^n folded into the term's running product
                const size_t ro = (size_t)slot * a.real_stride;
#pragma unroll 1
                for (int i = t; i < nrow * N; i += nthr) {
                    const int rl = i / N, x = i - rl * N;
                    const C z = Z[(rl & (G - 1)) * SF + spad(x)];
                    const size_t idx = ro + real_row_offset(sp, r0 + rl) + x;
                    const T v = ipow<T>(rl < G ? z.x : z.y, a.fac_power);
                    const T tp = a.fac_first_factor ? v : a.fac_tp[idx] * v;
                    if (a.fac_last_factor) a.fac_acc[idx] = a.fac_first_term ? tp : a.fac_acc[idx] + tp;
                    else a.fac_tp[idx] = tp;
                }
                return;
            }
            T *__restrict__ dst = a.real_out + (size_t)slot * a.real_stride;
#pragma unroll 1
            for (int i = t; i < nrow * N; i += nthr) {
                const int rl = i / N, x = i - rl * N;
                const C z = Z[(rl & (G - 1)) * SF + spad(x)];
                dst[real_row_offset(sp, r0 + rl) + x] = rl < G ? z.x : z.y;
            }
            return;
        }
        // forward transform of the real-space product (phi^d)^p of both rows
        // (ROW_ADJ: of p r^(p-1) s, with s the rows just transformed and r read
        // from real_in; ROW_FUSED with real_out: the rows are stored as well)
        const int p = fp.power;
        C *zf = Z + g * SF;
        C *other = (which == 0 ? B1 : B0) + g * SF;
        const bool adj = mode == ROW_ADJ;
        const T *ra = nullptr, *rb = nullptr;
        T *wa = nullptr, *wb = nullptr;
        if (adj) {
            const T *base = a.real_in + (size_t)slot * a.real_stride;
            if (g < nrow) ra = base + real_row_offset(sp, r0 + g);
            if (G + g < nrow) rb = base + real_row_offset(sp, r0 + G + g);
        } else if (a.real_out) {
            T *base = a.real_out + (size_t)slot * a.real_stride;
            if (g < nrow) wa = base + real_row_offset(sp, r0 + g);
            if (G + g < nrow) wb = base + real_row_offset(sp, r0 + G + g);
        }
        const int which2 = fft_run<T, N, EMAX, -1>(
            [&](int k) {
                const C z = zf[spad(k)];
                if (adj) {
                    const T xa = ra ? ra[k] : T(0), xb = rb ? rb[k] : T(0);
                    return mk<T>(T(p) * ipow<T>(xa, p - 1) * z.x, T(p) * ipow<T>(xb, p - 1) * z.y);
                }
                if (wa) wa[k] = z.x;
                if (wb) wb[k] = z.y;
                return mk<T>(ipow<T>(z.x, p), ipow<T>(z.y, p));
            },
            smem_sink, other, zf, lane, active, tw);
        R = which2 == 0 ? (which == 0 ? B1 : B0) : (which == 0 ? B0 : B1);
    }
    __syncthreads();
    // ---- split the pairs and write the half spectra of all tiles (coalesced)
    C *__restrict__ dst = a.out + sofs;
    const int logG2 = logG + 1;
#pragma unroll 1
    for (int i = t; i < sp.ntiles * G2 * W; i += nthr) {
        const int cc = i & 3, rl = (i >> 2) & (G2 - 1), tl = i >> (2 + logG2);
        if (rl >= nrow) continue;
        const int kx = tl * W + cc;
        C val = mk<T>(0, 0);
        if (kx <= N / 2) {
            const C *rb = R + (rl & (G - 1)) * SF;
            const C wk = rb[spad(kx)];
            const C wm = rb[spad((N - kx) & (N - 1))];
            val = rl < G ? mk<T>(T(0.5) * (wk.x + wm.x), T(0.5) * (wk.y - wm.y))
                         : mk<T>(T(0.5) * (wk.y + wm.y), T(-0.5) * (wk.x - wm.x));
        }
        dst[((size_t)tl * rows + r0 + rl) * W + cc] = val;
    }
    if (a.inc_step && blockIdx.x == 0 && blockIdx.y == 0 && t == 0) *a.d_step += 1;
}

// ---------------------------------------------------------------------------
// k_mid: FFTs along y in 3D (N = ny points) for one tile and PZ z-planes,
// F = PZ W FFTs.  Threads: FFT f = t mod F, lane t / F.  Shared memory: S
// (the staged [ky][F] input; also a work buffer), B0.
// ---------------------------------------------------------------------------
template <typename T, int N> struct MidSmem {
    __host__ __device__ static int s_elems(int F) {
        const int a = N * F, b = F * sf_fft_fastest(N, F);
        return a > b ? a : b;
    }
    __host__ __device__ static size_t bytes(int F) {
        return 128 + sizeof(cplx<T>) * ((size_t)twiddle_elems<N>() + (size_t)s_elems(F) + (size_t)F * sf_fft_fastest(N, F));
    }
};

template <typename T, int N, int EMAX>
__global__ void __launch_bounds__(256) k_mid(const MidArgs<T> a) {
    using C = cplx<T>;
    using L = MidSmem<T, N>;
    constexpr int TPF = FftShape<N, EMAX>::TPF;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);
    const SysP<T> &sp = a.sp;
    const int F = a.PZ * W;
    const int logF = __ffs(F) - 1;
    const int SF = sf_fft_fastest(N, F);
    C *TW = reinterpret_cast<C *>(smem_raw + 128);             // roots of unity of length N
    C *S = TW + twiddle_elems<N>();
    C *B0 = S + L::s_elems(F);
    const int slot = a.slot0 + blockIdx.z;
    const size_t sofs = (size_t)slot * a.slot_stride;
    const int t = threadIdx.x, nthr = blockDim.x;
    const int tile = blockIdx.x;
    const int pos0 = blockIdx.y * a.PZ;
    const int nz = sp.nz;
    const bool masked_in = a.mode == MID_INV_MASK;
    const int kmy = a.fps[slot].kmax[1];
    const C *__restrict__ src = a.in + sofs;
    const uint32_t seg = (uint32_t)(F * sizeof(C));
    pdl_wait();
    pdl_trigger();
    if (t == 0) {
        int n = 0;
        for (int o = 0; o < N; ++o) n += (!masked_in || abs(signed_k(o, N)) <= kmy) ? 1 : 0;
        mbar_init(bar, 1);
        mbar_expect_tx(bar, seg * n + twiddle_bytes<C, N>());
        if (twiddle_bytes<C, N>()) bulk_g2s(TW, a.tw + twiddle_offset(N, EMAX), twiddle_bytes<C, N>(), bar);
    }
    __syncthreads();
    for (int o = t; o < N; o += nthr) {
        if (!masked_in || abs(signed_k(o, N)) <= kmy)
            bulk_g2s(S + o * F, src + (((size_t)tile * N + o) * nz + pos0) * W, seg, bar);
    }
    if (masked_in)
        for (int i = t; i < N * F; i += nthr)
            if (abs(signed_k(i >> logF, N)) > kmy) S[i] = mk<T>(0, 0);
    if (!mbar_wait_all(bar, 0, a.d_status)) return;
    const int f = t & (F - 1), lane = t >> logF;
    const bool active = lane < TPF;
    C *__restrict__ dst = a.out + sofs + (((size_t)tile * N) * nz + pos0) * W + f;
    const size_t ostride = (size_t)nz * W;
    auto src_f = [&](int p) { return S[p * F + f]; };
    auto sink = [&](int p, C v, C *) { dst[p * ostride] = v; };
    const C *__restrict__ tw = TW;
    if (a.mode == MID_FWD) fft_run<T, N, EMAX, -1>(src_f, sink, B0 + f * SF, S + f * SF, lane, active, tw);
    else fft_run<T, N, EMAX, +1>(src_f, sink, B0 + f * SF, S + f * SF, lane, active, tw);
    if (a.inc_step && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && t == 0) *a.d_step += 1;
}

// ---------------------------------------------------------------------------
// auxiliary kernels (set-up and output; not on the per-step path)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_init_uniform(T *real, long long nsites, T lo, T hi, uint32_t s0, uint32_t s1, int field_id) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nsites;
         i += (long long)gridDim.x * blockDim.x) {
        const u32x4 r = philox4x32_10(u32x4{(uint32_t)i, 0u, (uint32_t)field_id, 1u}, s0, s1);
        real[i] = lo + (hi - lo) * uniform24<T>(r.x);
    }
}

// Q = (first ? 0 : Q) + M(q) Pt over one slot's tiled spectrum, M(q) = sum_p m_p (q^2)^p
template <typename T>
__global__ void k_combine(const SysP<T> sp, cplx<T> *Q, const cplx<T> *Pt, T m0, T m1, T m2, T m3, T m4, int first) {
    const long long n = (long long)sp.ntiles * sp.rows * W;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % W);
        const long long tr = i / W;
        const int row = (int)(tr % sp.rows), tile = (int)(tr / sp.rows);
        const int kx = tile * W + c;
        const int ky = sp.dim == 3 ? row / sp.nz : (sp.dim == 2 ? row : 0);
        const int kz = sp.dim == 3 ? row % sp.nz : 0;
        const T qx = T(kx) * sp.gx, qy = T(signed_k(ky, sp.ny)) * sp.gy, qz = T(signed_k(kz, sp.nz)) * sp.gz;
        const T q2 = qx * qx + qy * qy + qz * qz;
        const T M = m0 + q2 * (m1 + q2 * (m2 + q2 * (m3 + q2 * m4)));
        const cplx<T> p = Pt[i];
        const cplx<T> base = first ? mk<T>(0, 0) : Q[i];
        Q[i] = kx < sp.hx ? mk<T>(base.x + M * p.x, base.y + M * p.y) : mk<T>(0, 0);
    }
}

// Boundary frame along x of a real field [rows][nx]: x < w takes lo, x >= nx - w takes hi.
template <typename T> __global__ void k_frame(T *real, int nx, long long rows, int w, T lo, T hi) {
    const long long n = rows * (2LL * w);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / (2 * w);
        const int j = (int)(i - r * (2 * w));
        const int x = j < w ? j : nx - 2 * w + j;
        real[r * nx + x] = j < w ? lo : hi;
    }
}

template <typename T>
__global__ void k_tiles_half(SysP<T> sp, cplx<T> *tiles, cplx<T> *half, int to_half) {
    const long long n = (long long)sp.nz * sp.ny * sp.hx;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int kx = (int)(i % sp.hx);
        const long long r2 = i / sp.hx;
        const int ky = (int)(r2 % sp.ny), kz = (int)(r2 / sp.ny);
        const int row = sp.dim == 3 ? ky * sp.nz + kz : ky;
        const size_t ti = ((size_t)(kx / W) * sp.rows + row) * W + kx % W;
        if (to_half) half[i] = tiles[ti];
        else tiles[ti] = half[i];
    }
}

// Start of a recomputed adjoint segment j = *d_seg (read on the device, so that
// one captured graph serves every segment): checkpoint j -> dst, and the step
// counters of its first step.
template <typename T>
__global__ void k_segment_begin(cplx<T> *dst, const cplx<T> *ck, size_t slot_elems, const long long *d_seg,
                                long long step_base, long long K, long long *d_step, long long *d_adj_base) {
    const long long j = *d_seg;
    const cplx<T> *src = ck + (size_t)j * slot_elems;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < slot_elems; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *d_step = step_base + j * K;
        *d_adj_base = step_base + j * K;
    }
}

template <typename T>
cudaError_t launch_segment_begin(cplx<T> *dst, const cplx<T> *ck, size_t slot_elems, const long long *d_seg,
                                 long long step_base, long long K, long long *d_step, long long *d_adj_base,
                                 cudaStream_t st) {
    long long blocks = (long long)((slot_elems + 255) / 256);
    if (blocks > 1184) blocks = 1184;
    k_segment_begin<T><<<(int)blocks, 256, 0, st>>>(dst, ck, slot_elems, d_seg, step_base, K, d_step, d_adj_base);
    return cudaGetLastError();
}

// S(q) accumulation: acc[0..nbins) sum S, acc[nbins..2nbins) counts,
// acc[2nbins] sum S, acc[2nbins+1] sum |q| S.  Bin arithmetic in FP64 with
// explicit round-to-nearest operations (no contraction).
template <typename T>
__global__ void k_structure_factor(SysP<T> sp, double dx0, double dx1, double dx2, const cplx<T> *tiles,
                                   int nbins, double *acc) {
    extern __shared__ double sacc[];
    for (int i = threadIdx.x; i < 2 * nbins + 2; i += blockDim.x) sacc[i] = 0.0;
    __syncthreads();
    const long long n = (long long)sp.nz * sp.ny * sp.hx;
    const double inv_ns = 1.0 / ((double)sp.nx * sp.ny * sp.nz);
    const double dxs[3] = {dx0, dx1, dx2};
    const int Ns[3] = {sp.nx, sp.ny, sp.nz};
    const int lane = threadIdx.x & 31;
    double tS = 0.0, tQ = 0.0;   // the thread's share of the two totals
    // the warps step through the modes 32 at a time (neighbouring kx of one row, a
    // handful of bins at most): lanes in one bin are summed with shuffles and one
    // lane adds the sums to the CTA's bins
    for (long long i0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); i0 < n;
         i0 += (long long)gridDim.x * blockDim.x) {
        const long long i = i0 + lane;
        int b = -1;
        double vS = 0.0, vW = 0.0;
        if (i < n) {
            const int kx = (int)(i % sp.hx);
            const long long r2 = i / sp.hx;
            const int ky = (int)(r2 % sp.ny), kz = (int)(r2 / sp.ny);
            const int ks[3] = {kx, signed_k(ky, sp.ny), signed_k(kz, sp.nz)};
            double s2 = 0.0, qq = 0.0;
            for (int j = 0; j < 3; ++j) {
                if (Ns[j] == 1) continue;
                const double num = __dmul_rn(__dmul_rn(__dmul_rn(2.0, (double)nbins), (double)ks[j]), dx0);
                const double tj = __ddiv_rn(num, __dmul_rn((double)Ns[j], dxs[j]));
                s2 = __dadd_rn(s2, __dmul_rn(tj, tj));
                const double qj = 6.283185307179586 * ks[j] / (Ns[j] * dxs[j]);
                qq += qj * qj;
            }
            const double s = __dsqrt_rn(s2);
            if (s2 != 0.0 && s <= (double)nbins) {
                b = (int)ceil(s) - 1;
                const int row = sp.dim == 3 ? ky * sp.nz + kz : ky;
                const cplx<T> z = tiles[((size_t)(kx / W) * sp.rows + row) * W + kx % W];
                const double S = ((double)z.x * z.x + (double)z.y * z.y) * inv_ns;
                vW = (kx == 0 || 2 * kx == sp.nx) ? 1.0 : 2.0;
                vS = vW * S;
                tS += vS;
                tQ += vW * sqrt(qq) * S;
            }
        }
        unsigned todo = __ballot_sync(0xffffffffu, b >= 0);
        while (todo) {
            const int src = __ffs(todo) - 1;
            const int b0 = __shfl_sync(0xffffffffu, b, src);
            const bool mine = b == b0;
            double sv = mine ? vS : 0.0, wv = mine ? vW : 0.0;
            for (int o = 16; o > 0; o >>= 1) {
                sv += __shfl_xor_sync(0xffffffffu, sv, o);
                wv += __shfl_xor_sync(0xffffffffu, wv, o);
            }
            if (lane == src) {
                atomicAdd(&sacc[b0], sv);
                atomicAdd(&sacc[nbins + b0], wv);
            }
            todo &= ~__ballot_sync(0xffffffffu, mine);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        tS += __shfl_xor_sync(0xffffffffu, tS, o);
        tQ += __shfl_xor_sync(0xffffffffu, tQ, o);
    }
    if (lane == 0) {
        if (tS != 0.0) atomicAdd(&sacc[2 * nbins], tS);
        if (tQ != 0.0) atomicAdd(&sacc[2 * nbins + 1], tQ);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 2 * nbins + 2; i += blockDim.x)
        if (sacc[i] != 0.0) atomicAdd(&acc[i], sacc[i]);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
// launch with programmatic stream serialisation (PDL)
template <class K, class A>
cudaError_t launch_pdl(K kernel, dim3 grid, int threads, size_t smem, cudaStream_t st, const A &args) {
    if (!args.sp.pdl) {
        kernel<<<grid, threads, smem, st>>>(args);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args);
}

template <class K> cudaError_t ensure_smem(K kernel, size_t smem) {
    if (smem <= 48 * 1024) return cudaSuccess;
    if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <typename T, int N, int EMAX>
cudaError_t launch_col_n(const ColArgs<T> &a, int nf, int gx, int gy, cudaStream_t st) {
    const int threads = col_threads(N, EMAX, a.F);
    const bool adj = a.mode == COL_ADJ_A || a.mode == COL_ADJ_B || a.mode == COL_ADJ_BA;
    const size_t smem = a.mode == COL_ADJ_BA ? ColSmem<T, N>::bytes_adj(a.F) : ColSmem<T, N>::bytes(a.F);
    if (a.F * FftShape<N, EMAX>::TPF > 512 || (a.F & (a.F - 1)) != 0 || a.F % W != 0)
        return cudaErrorInvalidConfiguration;
    cudaError_t e = adj ? ensure_smem(k_col<T, N, EMAX, true>, smem) : ensure_smem(k_col<T, N, EMAX, false>, smem);
    if (e != cudaSuccess) return e;
    if (adj) return launch_pdl(k_col<T, N, EMAX, true>, dim3(gx, gy, nf), threads, smem, st, a);
    return launch_pdl(k_col<T, N, EMAX, false>, dim3(gx, gy, nf), threads, smem, st, a);
}

template <typename T, int EMAX>
cudaError_t launch_col_e(const ColArgs<T> &a, int nf, int gx, int gy, cudaStream_t st) {
    switch (a.sp.n_inner) {
        case 1: return launch_col_n<T, 1, EMAX>(a, nf, gx, gy, st);
        case 4: return launch_col_n<T, 4, EMAX>(a, nf, gx, gy, st);
        case 8: return launch_col_n<T, 8, EMAX>(a, nf, gx, gy, st);
        case 16: return launch_col_n<T, 16, EMAX>(a, nf, gx, gy, st);
        case 32: return launch_col_n<T, 32, EMAX>(a, nf, gx, gy, st);
        case 64: return launch_col_n<T, 64, EMAX>(a, nf, gx, gy, st);
        case 128: return launch_col_n<T, 128, EMAX>(a, nf, gx, gy, st);
        case 256: return launch_col_n<T, 256, EMAX>(a, nf, gx, gy, st);
        case 512: return launch_col_n<T, 512, EMAX>(a, nf, gx, gy, st);
        case 1024: return launch_col_n<T, 1024, EMAX>(a, nf, gx, gy, st);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T, int EMAX> size_t col_smem_bytes_e(int n_inner, int F, int mode) {
    const bool two = mode == COL_ADJ_BA;
    switch (n_inner) {
#define PSS_COL_SMEM(n) case n: return two ? ColSmem<T, n>::bytes_adj(F) : ColSmem<T, n>::bytes(F);
        PSS_COL_SMEM(1) PSS_COL_SMEM(4) PSS_COL_SMEM(8) PSS_COL_SMEM(16) PSS_COL_SMEM(32) PSS_COL_SMEM(64)
        PSS_COL_SMEM(128) PSS_COL_SMEM(256) PSS_COL_SMEM(512) PSS_COL_SMEM(1024)
#undef PSS_COL_SMEM
        default: return 0;
    }
}

template <typename T, int N, int EMAX> cudaError_t launch_row_n(const RowArgs<T> &a, int nf, cudaStream_t st) {
    const int G = a.G;
    const int threads = G * FftShape<N, EMAX>::TPF < 32 ? 32 : G * FftShape<N, EMAX>::TPF;
    const size_t smem = RowSmem<T, N>::bytes(G, a.sp.ntiles);
    if (threads > 256 || (G & (G - 1)) != 0) return cudaErrorInvalidConfiguration;
    cudaError_t e = ensure_smem(k_row<T, N, EMAX>, smem);
    if (e != cudaSuccess) return e;
    const int grid = (a.sp.rows + 2 * G - 1) / (2 * G);
    return launch_pdl(k_row<T, N, EMAX>, dim3(grid, nf), threads, smem, st, a);
}

template <typename T, int EMAX> cudaError_t launch_row_e(const RowArgs<T> &a, int nf, cudaStream_t st) {
    switch (a.sp.nx) {
        case 4: return launch_row_n<T, 4, EMAX>(a, nf, st);
        case 8: return launch_row_n<T, 8, EMAX>(a, nf, st);
        case 16: return launch_row_n<T, 16, EMAX>(a, nf, st);
        case 32: return launch_row_n<T, 32, EMAX>(a, nf, st);
        case 64: return launch_row_n<T, 64, EMAX>(a, nf, st);
        case 128: return launch_row_n<T, 128, EMAX>(a, nf, st);
        case 256: return launch_row_n<T, 256, EMAX>(a, nf, st);
        case 512: return launch_row_n<T, 512, EMAX>(a, nf, st);
        case 1024: return launch_row_n<T, 1024, EMAX>(a, nf, st);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T, int N, int EMAX>
cudaError_t launch_mid_n(const MidArgs<T> &a, int nf, int n_tiles, cudaStream_t st) {
    const int F = a.PZ * W;
    const int threads = F * FftShape<N, EMAX>::TPF < 32 ? 32 : F * FftShape<N, EMAX>::TPF;
    const size_t smem = MidSmem<T, N>::bytes(F);
    if (threads > 256 || (F & (F - 1)) != 0) return cudaErrorInvalidConfiguration;
    cudaError_t e = ensure_smem(k_mid<T, N, EMAX>, smem);
    if (e != cudaSuccess) return e;
    return launch_pdl(k_mid<T, N, EMAX>, dim3(n_tiles, a.sp.nz / a.PZ, nf), threads, smem, st, a);
}

template <typename T, int EMAX>
cudaError_t launch_mid_e(const MidArgs<T> &a, int nf, int n_tiles, cudaStream_t st) {
    switch (a.sp.ny) {
        case 4: return launch_mid_n<T, 4, EMAX>(a, nf, n_tiles, st);
        case 8: return launch_mid_n<T, 8, EMAX>(a, nf, n_tiles, st);
        case 16: return launch_mid_n<T, 16, EMAX>(a, nf, n_tiles, st);
        case 32: return launch_mid_n<T, 32, EMAX>(a, nf, n_tiles, st);
        case 64: return launch_mid_n<T, 64, EMAX>(a, nf, n_tiles, st);
        case 128: return launch_mid_n<T, 128, EMAX>(a, nf, n_tiles, st);
        case 256: return launch_mid_n<T, 256, EMAX>(a, nf, n_tiles, st);
        case 512: return launch_mid_n<T, 512, EMAX>(a, nf, n_tiles, st);
        case 1024: return launch_mid_n<T, 1024, EMAX>(a, nf, n_tiles, st);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t launch_init_uniform(T *real, long long nsites, double lo, double hi, uint64_t seed, int field_id,
                                cudaStream_t st) {
    const int threads = 256;
    long long blocks = (nsites + threads - 1) / threads;
    if (blocks > 65535) blocks = 65535;
    k_init_uniform<T><<<(int)blocks, threads, 0, st>>>(real, nsites, T(lo), T(hi), (uint32_t)(seed & 0xffffffffu),
                                                     (uint32_t)(seed >> 32), field_id);
    return cudaGetLastError();
}

static inline int aux_blocks(long long n) {
    long long blocks = (n + 255) / 256;
    return (int)(blocks > 65535 ? 65535 : (blocks < 1 ? 1 : blocks));
}

template <typename T>
cudaError_t launch_combine(const SysP<T> &sp, cplx<T> *Q, const cplx<T> *Pt, const double *m, int first,
                           cudaStream_t st) {
    k_combine<T><<<aux_blocks((long long)sp.ntiles * sp.rows * W), 256, 0, st>>>(
        sp, Q, Pt, T(m[0]), T(m[1]), T(m[2]), T(m[3]), T(m[4]), first);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_frame(T *real, int nx, long long rows, int width, double lo, double hi, cudaStream_t st) {
    if (width < 1 || 2 * width > nx) return cudaErrorInvalidValue;
    const long long n = rows * 2LL * width;
    long long blocks = (n + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    k_frame<T><<<(int)blocks, 256, 0, st>>>(real, nx, rows, width, T(lo), T(hi));
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_tiles_to_half(const SysP<T> &sp, const cplx<T> *tiles, cplx<T> *half, cudaStream_t st) {
    const long long n = (long long)sp.nz * sp.ny * sp.hx;
    long long blocks = (n + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    k_tiles_half<T><<<(int)blocks, 256, 0, st>>>(sp, const_cast<cplx<T> *>(tiles), half, 1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_half_to_tiles(const SysP<T> &sp, const cplx<T> *half, cplx<T> *tiles, cudaStream_t st) {
    const long long n = (long long)sp.nz * sp.ny * sp.hx;
    long long blocks = (n + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    k_tiles_half<T><<<(int)blocks, 256, 0, st>>>(sp, tiles, const_cast<cplx<T> *>(half), 0);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_structure_factor(const SysP<T> &sp, const double dx[3], const cplx<T> *tiles, int nbins,
                                    double *acc, cudaStream_t st) {
    const long long n = (long long)sp.nz * sp.ny * sp.hx;
    // at most 512 CTAs: each adds its 2 nbins + 2 sums to the same global words
    long long blocks = (n + 255) / 256;
    if (blocks > 512) blocks = 512;
    const size_t smem = sizeof(double) * (size_t)(2 * nbins + 2);
    cudaError_t e = ensure_smem(k_structure_factor<T>, smem);
    if (e != cudaSuccess) return e;
    k_structure_factor<T><<<(int)blocks, 256, smem, st>>>(sp, dx[0], dx[1], dx[2], tiles, nbins, acc);
    return cudaGetLastError();
}

// the step kernels of one precision and FFT radix cap
#define PSS_INSTANTIATE_STEP(T, EMAX)                                                                       \
    template cudaError_t launch_col_e<T, EMAX>(const ColArgs<T> &, int, int, int, cudaStream_t);           \
    template size_t col_smem_bytes_e<T, EMAX>(int, int, int);                                              \
    template cudaError_t launch_row_e<T, EMAX>(const RowArgs<T> &, int, cudaStream_t);                     \
    template cudaError_t launch_mid_e<T, EMAX>(const MidArgs<T> &, int, int, cudaStream_t);

// the auxiliary kernels of one precision
#define PSS_INSTANTIATE_AUX(T)                                                                               \
    template cudaError_t launch_init_uniform<T>(T *, long long, double, double, uint64_t, int, cudaStream_t); \
    template cudaError_t launch_tiles_to_half<T>(const SysP<T> &, const cplx<T> *, cplx<T> *, cudaStream_t); \
    template cudaError_t launch_frame<T>(T *, int, long long, int, double, double, cudaStream_t);              \
    template cudaError_t launch_combine<T>(const SysP<T> &, cplx<T> *, const cplx<T> *, const double *, int,  \
                                           cudaStream_t);                                                   \
    template cudaError_t launch_half_to_tiles<T>(const SysP<T> &, const cplx<T> *, cplx<T> *, cudaStream_t); \
    template cudaError_t launch_segment_begin<T>(cplx<T> *, const cplx<T> *, size_t, const long long *, long long, \
                                                 long long, long long *, long long *, cudaStream_t);             \
    template cudaError_t launch_structure_factor<T>(const SysP<T> &, const double *, const cplx<T> *, int,   \
                                                    double *, cudaStream_t);

}  // namespace pss

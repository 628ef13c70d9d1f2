// pss_adj2d.cuh -- the column part of the adjoint step on FFT groups (FP32 2D,
// sides of 256, 512 or 1024 points), arXiv:2405.02410, Eq. timeupdate.
//
// For a fixed noise realisation the step phi' = H[g (phi + dt M P + xi)] has
// the adjoint recursion (the oracle's orc_adjoint writes it on the full
// spectrum in FP64):
//   part A: mu = g lambda', the gradient sums of the implicit and explicit
//           coefficients and of the noise strength, nu = dt M mu transformed
//           back along y (all columns);
//   part B: lambda = mu + m F[w] / N (F[w]: the adjoint's x pass transformed
//           along y), Hermitian part on the kx = 0, Nx/2 columns;
//   part BA: part B of step n, then part A of step n - 1 on the lambda it
//           left, without lambda going through global memory.
// k2_col_adj takes one pair of neighbouring columns (kx = 2u, 2u + 1: one
// Philox call draws the noise of both) per CTA: its two FFT groups transform
// one column each, and every thread of the CTA (the groups and as many
// helper threads) joins the element-wise parts, so that a 2D side of
// 256..1024 points spreads over (Nx/2 + 2)/2 CTAs (the generic column
// kernel takes 4 columns per CTA: 33 CTAs at 256^2).  Argument semantics are those of the generic kernel's
// adjoint modes (ColArgs): the adjoint field and the forward state after the
// step are tiled, the x-transformed w is tiled (the x pass's output), the
// products of the recomputed steps are column-major.  The transforms are the
// group FFTs of pss_fast2d.cuh; an inverse is conj(F(conj x)).
#pragma once

#include "pss_fast2d.cuh"

namespace pss {

// Shared memory: roots of unity | per group (column) two transform buffers
// and the column's adjoint field (lambda / mu, natural order).
template <int N, int E> struct Adj2Shape {
    using S = GShape<N, E>;
    static constexpr int THREADS = 4 * S::TPF;        // 2 FFT groups and as many helper threads
    static constexpr int WS = 2 * S::BUF + N + 4;    // per column
    static constexpr size_t TW = 0;
    static constexpr size_t GB = TW + sizeof(float2) * N;
    static constexpr size_t BYTES = GB + sizeof(float2) * 2 * WS;
};

template <int N, int E>
__global__ void __launch_bounds__(Adj2Shape<N, E>::THREADS) k2_col_adj(const ColArgs<float> a) {
    using C = float2;
    using S = GShape<N, E>;
    using L = Adj2Shape<N, E>;
    constexpr int TPF = S::TPF, NT = L::THREADS;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    C *TW = reinterpret_cast<C *>(smem_raw + L::TW);
    C *GBUF = reinterpret_cast<C *>(smem_raw + L::GB);
    __shared__ FieldP<float> sfp;
    __shared__ double red[11];
    const SysP<float> &sp = a.sp;
    const FieldP<float> &fp = sfp;
    const int t = threadIdx.x;
    const int g = t / TPF, gl = t - g * TPF;   // FFT group g < 2 (column kx0 + g); g >= 2: a helper thread
    const int slot = a.slot0 + blockIdx.y;
    const size_t so = (size_t)slot * a.slot_stride;
    const int kx0 = 2 * blockIdx.x;            // the CTA's column pair
    for (int i = t; i < (int)(sizeof(FieldP<float>) / 4); i += NT)
        reinterpret_cast<uint32_t *>(&sfp)[i] = reinterpret_cast<const uint32_t *>(&a.fps[slot])[i];
    for (int i = t; i < N; i += NT) TW[i] = a.tw[twiddle_offset(N, E) + i];
    if (t < 11) red[t] = 0.0;
    const int mode = a.mode;
    const bool do_b = mode != COL_ADJ_A, do_a = mode != COL_ADJ_B;
    constexpr bool ODD = GShape<N, E>::NPASS % 2 == 1;   // a forward transform's result is in b0
    // column c (0, 1) of the pair: buffers, adjoint field, the transform's result P and the free buffer
    auto b0_of = [&](int c) { return GBUF + (size_t)c * L::WS; };
    auto b1_of = [&](int c) { return b0_of(c) + S::BUF; };
    auto x3_of = [&](int c) { return b1_of(c) + S::BUF; };
    auto p_of = [&](int c) { return ODD ? b0_of(c) : b1_of(c); };
    auto nu_of = [&](int c) { return ODD ? b1_of(c) : b0_of(c); };
    // element ky of column kx in a tiled array of this slot; of a column-major one
    auto tiled = [&](int kx, int ky) { return so + ((size_t)(kx >> 2) * N + ky) * 4 + (kx & 3); };
    auto colmaj = [&](int kx, int ky) { return so + (size_t)kx * N + ky; };
    const bool v0 = kx0 < sp.hx, v1 = kx0 + 1 < sp.hx;   // columns past Nx/2 are not transformed

    // every thread: the adjoint field and the first column to transform (F[w], tiled,
    // for parts B and BA; the product, column-major, for A) of both columns.  Each
    // loop issues all of a thread's loads before its first shared-memory store, so
    // that their L2 round trips overlap (PER elements per thread)
    constexpr int PER = 2 * N / NT;
    {
        C vs[PER], vi[PER];
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int i = t + u * NT, c = i / N, ky = i - c * N, kx = kx0 + c;
            vs[u] = vi[u] = mk<float>(0.f, 0.f);
            if (kx < sp.hx) {
                vs[u] = __ldcg(a.state + tiled(kx, ky));
                vi[u] = __ldcg(a.in + (a.in_colmajor ? colmaj(kx, ky) : tiled(kx, ky)));
            }
        }
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int i = t + u * NT, c = i / N, ky = i - c * N;
            x3_of(c)[ky] = vs[u];
            b1_of(c)[ky] = vi[u];
        }
    }
    __syncthreads();
    auto transform = [&]() {   // each group: forward transform of its column's b1 -> P
        if (g < 2 && (g == 0 ? v0 : v1)) fft_fwd_group<N, E>(b1_of(g), b0_of(g), b1_of(g), gl, 1 + g, TW, 0);
        __syncthreads();
    };
    transform();
    if (do_b) {
        // lambda = mu + m F[w] / N on the kept modes
        for (int i = t; i < 2 * N; i += NT) {
            const int c = i / N, ky = i - c * N, kx = kx0 + c;
            if (kx >= sp.hx) continue;
            const bool keep = kx <= fp.kmax[0] && abs(signed_k(ky, N)) <= fp.kmax[1];
            C *x3 = x3_of(c);
            const C mu = x3[ky], pv = p_of(c)[ky];
            x3[ky] = keep ? mk<float>(mu.x + pv.x * sp.inv_nsites, mu.y + pv.y * sp.inv_nsites) : mu;
        }
        __syncthreads();
        // Hermitian part of lambda on the kx = 0, Nx/2 columns
        for (int c = 0; c < 2; ++c) {
            const int kx = kx0 + c;
            if (kx >= sp.hx || (kx != 0 && 2 * kx != sp.nx)) continue;
            C *x3 = x3_of(c);
            for (int pos = t; pos < N / 2 + 1; pos += NT) {
                const int ppos = (N - pos) & (N - 1);
                const C u0 = x3[pos], u1 = x3[ppos];
                const C h = mk<float>(0.5f * (u0.x + u1.x), 0.5f * (u0.y - u1.y));
                x3[pos] = h;
                x3[ppos] = mk<float>(h.x, -h.y);
            }
        }
        __syncthreads();
        if (mode == COL_ADJ_BA) {
            // the A part's P: forward transform of the earlier step's product
            C vz[PER];
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                const int i = t + u * NT, c = i / N, ky = i - c * N, kx = kx0 + c;
                vz[u] = kx < sp.hx ? __ldcg(a.in2 + (a.in2_colmajor ? colmaj(kx, ky) : tiled(kx, ky)))
                                   : mk<float>(0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                const int i = t + u * NT, c = i / N, ky = i - c * N;
                b1_of(c)[ky] = vz[u];
            }
            __syncthreads();
            transform();
        }
    }

    // part A: mu = g lambda, gradient sums, conj(nu) into the free buffer; one
    // Philox draw per ky serves both columns
    float acc[11];
#pragma unroll
    for (int i = 0; i < 11; ++i) acc[i] = 0.f;
    if (do_a) {
        const uint32_t step = (uint32_t)(a.adj_step + (a.d_adj_base ? *a.d_adj_base : 0));
        const PhiloxKey key = philox_key(fp.seed_lo, fp.seed_hi);
        const float qe = float(kx0) * sp.gx, qo = float(kx0 + 1) * sp.gx;
        // the forward state after the step at the thread's modes, all loads in flight together
        constexpr int PKY = N / NT;   // rows per thread
        C ph[PKY][2];
#pragma unroll
        for (int u = 0; u < PKY; ++u)
#pragma unroll
            for (int c = 0; c < 2; ++c)
                ph[u][c] = kx0 + c < sp.hx ? __ldcg(a.aux + tiled(kx0 + c, t + u * NT)) : mk<float>(0.f, 0.f);
#pragma unroll
        for (int u = 0; u < PKY; ++u) {
            const int ky = t + u * NT;
            if (!v0) break;
            const float qy = float(signed_k(ky, N)) * sp.gy;
            const float q2c[2] = {qe * qe + qy * qy, qo * qo + qy * qy};
            C xin[2] = {mk<float>(0.f, 0.f), mk<float>(0.f, 0.f)};
            if (fp.noisy)
                noise_pair<float>(kx0 == 0 || 2 * kx0 == sp.nx, kx0, ky, 0,
                                  noise_amp<float>(fp.sigma0, fp.noise_pow, q2c[0]),
                                  noise_amp<float>(fp.sigma0, fp.noise_pow, q2c[1]), v1, sp, (uint32_t)fp.field_id,
                                  key, step, xin[0], xin[1]);
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int kx = kx0 + c;
                if (kx >= sp.hx) continue;
                const float q2 = q2c[c];
                const C pv = p_of(c)[ky];
                const float gg = 1.f / (1.f + sp.dt * poly5<float>(fp.O, q2));
                C *x3 = x3_of(c);
                const C mu = cscale<float>(x3[ky], gg);
                x3[ky] = mu;
                const float dtM = fp.power > 0 ? sp.dt * poly5<float>(fp.M, q2) : 0.f;
                nu_of(c)[ky] = mk<float>(mu.x * dtM, -mu.y * dtM);   // conj(nu)
                const float wgt = (kx == 0 || 2 * kx == sp.nx) ? 1.f : 2.f;
                const C phin = ph[u][c];
                const float a_phi = wgt * sp.dt * (mu.x * phin.x + mu.y * phin.y);
                const float a_P = wgt * sp.dt * (mu.x * pv.x + mu.y * pv.y);
                float q2k = 1.f;
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    acc[k] -= q2k * a_phi;
                    acc[5 + k] += q2k * a_P;
                    q2k *= q2;
                }
                if (fp.noisy) acc[10] += wgt * (mu.x * xin[c].x + mu.y * xin[c].y);
            }
        }
    }
    __syncthreads();
    // the adjoint field (mu, or lambda after part B alone) back to the tiled array
    for (int i = t; i < 2 * N; i += NT) {
        const int c = i / N, ky = i - c * N, kx = kx0 + c;
        if (kx < sp.hx) a.state[tiled(kx, ky)] = x3_of(c)[ky];
    }
    if (do_a) {
        // CTA sum of the gradient terms: each warp's compensated FP32 sum (TwoSum) goes
        // to FP64 once, then one FP64 atomic per value and CTA
#pragma unroll
        for (int k = 0; k < 11; ++k) {
            float hi = acc[k], lo = 0.f;
            for (int o = 16; o > 0; o >>= 1) {
                const float ohi = __shfl_xor_sync(0xffffffffu, hi, o);
                const float olo = __shfl_xor_sync(0xffffffffu, lo, o);
                const float sm = __fadd_rn(hi, ohi), bp = __fsub_rn(sm, hi);
                const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(sm, bp)), __fsub_rn(ohi, bp));
                hi = sm;
                lo = __fadd_rn(__fadd_rn(lo, olo), err);
            }
            if ((t & 31) == 0) {
                const double v = (double)hi + (double)lo;
                if (v != 0.0) atomicAdd(&red[k], v);
            }
        }
        __syncthreads();
        if (t < 11 && red[t] != 0.0) atomicAdd(&a.grad[(size_t)slot * 11 + t], red[t]);
        // nu back along y (all columns): conj(F(conj nu)), stored tiled
        if (g < 2 && (g == 0 ? v0 : v1)) {
            const int kx = kx0 + g;
            fft_fwd_group_sink<N, E>(p_of(g), nu_of(g), gl, 1 + g, TW, [&](int q, C v) {
                a.out[tiled(kx, q)] = mk<float>(v.x, -v.y);
            });
        }
    }
}

}  // namespace pss

namespace pss {

// the adjoint's column part on FFT groups: one column pair per CTA
template <int N, int E>
cudaError_t launch_col2_adj_ne(const ColArgs<float> &a, int nslots, cudaStream_t st) {
    using L = Adj2Shape<N, E>;
    cudaError_t e = ensure_smem(k2_col_adj<N, E>, L::BYTES);
    if (e != cudaSuccess) return e;
    k2_col_adj<N, E><<<dim3((a.sp.hx + 1) / 2, nslots), L::THREADS, L::BYTES, st>>>(a);
    return cudaGetLastError();
}

}  // namespace pss

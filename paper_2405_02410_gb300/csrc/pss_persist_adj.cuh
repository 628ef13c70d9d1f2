// pss_persist_adj.cuh -- the backward pass of one recomputed segment of the
// FP32 2D adjoint as one persistent launch (arXiv:2405.02410, Eq. timeupdate;
// the adjoint recursion of k2_col_adj, pss_adj2d.cuh).
//
// For a fixed noise realisation the step phi' = H[g (phi + dt M P + xi)] is
// run backwards, from the segment's last step to its first:
//   column phase, part B of step i (i < len): lambda = mu + F_y[w] / N on the
//       kept modes (w: the x pass's result), Hermitian part on kx = 0, Nx/2;
//   column phase, part A of step i - 1 (or of the last step): mu = g lambda,
//       the gradient terms of the implicit and explicit coefficients and of
//       the noise strength, nu = dt M mu transformed back along y;
//   grid barrier; row phase, the x pass of step i - 1: C2R of nu's rows,
//       times p r^(p-1) (r: the step's stored real rows), R2C -> w;
//   grid barrier; and so on, ending with part B of the first step.
// Each CTA owns fixed columns (as k2p_step: up to two pairs kx = 2u, 2u + 1,
// one FFT group per column) and fixed row pairs.  In the column phase each
// group works on its own column, with its transforms chained through
// registers (pss_persist2d.cuh): the adjoint field of the CTA's columns stays
// in shared memory for the whole segment (it enters from the tiled array L
// and leaves to it at the end), the noise of each step is the one the
// segment's forward run stored, and each thread keeps compensated FP32 sums
// of its gradient terms over the segment, added up in FP64 at the end (warp,
// CTA, one FP64 atomic per value and CTA).  nu and w move through the tiled
// arrays NU and W between the phases.  The transforms and the element-wise
// recursion are those of k2_col_adj and of the adjoint x pass (k2_row in
// mode ROW_ADJ); the compiler may fuse their multiply-adds differently, so
// the two agree to FP32 rounding.  The grid barriers are those of k2p_step.
#pragma once

#include "pss_persist2d.cuh"

namespace pss {

// Shared memory: roots of unity (N) | adjoint field of the column slots [NG][N]
// | the groups' buffer pairs (row-phase placement of k2_row: WS apart) | the
// real rows of the row pairs [2 NG][N] (floats).
template <int N, int E> struct P2AdjShape {
    using S = GShape<N, E>;
    static constexpr int NG = 4;
    static constexpr int THREADS = NG * S::TPF;
    static constexpr size_t TW = 0;
    static constexpr size_t X3 = TW + sizeof(float2) * N;
    static constexpr size_t WB = X3 + sizeof(float2) * NG * N;
    static constexpr size_t MS = WB + sizeof(float2) * NG * S::WS;
    static constexpr size_t BYTES = MS + sizeof(float) * 2 * NG * N;
};

template <int N, int E>
__global__ void __launch_bounds__(P2AdjShape<N, E>::THREADS, 1) k2p_adj(const P2AdjArgs a) {
    using C = float2;
    using S = GShape<N, E>;
    using L = P2AdjShape<N, E>;
    constexpr int TPF = S::TPF, NG = L::NG, NT = L::THREADS, H = N / 2 + 1, UC = (H + 1) / 2;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    C *TW = reinterpret_cast<C *>(smem_raw + L::TW);
    C *X3 = reinterpret_cast<C *>(smem_raw + L::X3);   // adjoint field of slot c: X3[c N + ky]
    C *WB = reinterpret_cast<C *>(smem_raw + L::WB);
    float *MS = reinterpret_cast<float *>(smem_raw + L::MS);
    __shared__ FieldP<float> sfp;
    __shared__ double red[11];
    __shared__ int s_o2;
    __shared__ volatile int s_abort;
    const SysP<float> &sp = a.sp;
    const FieldP<float> &fp = sfp;
    const int t = threadIdx.x;
    const int g = t / TPF, gl = t - g * TPF;
    const unsigned nb = gridDim.x;
    int u0, u1, p0, p1;
    block_range(UC, (int)nb, blockIdx.x, u0, u1);
    block_range(N / 2, (int)nb, blockIdx.x, p0, p1);
    const int ncs = 2 * (u1 - u0), npr = p1 - p0;
    for (int i = t; i < (int)(sizeof(FieldP<float>) / 4); i += NT)
        reinterpret_cast<uint32_t *>(&sfp)[i] = reinterpret_cast<const uint32_t *>(a.fps)[i];
    for (int i = t; i < N; i += NT) TW[i] = a.tw[twiddle_offset(N, E) + i];
    if (t < 11) red[t] = 0.0;
    if (t == 0) {
        s_abort = ld_relaxed_gpu(&a.gs->abort) ? 1 : 0;   // an earlier launch gave up
    }
    // element ky of column kx in a tiled array ([kx / 4][ky][kx % 4])
    auto tiled = [&](int kx, int ky) { return ((size_t)(kx >> 2) * N + ky) * 4 + (kx & 3); };
    // the adjoint field of the CTA's columns (zero past Nx/2): all of a thread's loads
    // first, then the stores
    {
        constexpr int PX = NG * N / NT;
        C xv[PX];
#pragma unroll
        for (int q = 0; q < PX; ++q) {
            const int i = t + q * NT, c = i >> ilog2(N), ky = i & (N - 1), kx = 2 * u0 + c;
            xv[q] = i < ncs * N && kx < sp.hx ? __ldcg(a.L + tiled(kx, ky)) : mk<float>(0.f, 0.f);
        }
#pragma unroll
        for (int q = 0; q < PX; ++q)
            if (t + q * NT < ncs * N) X3[t + q * NT] = xv[q];
    }
    __syncthreads();
    if (s_abort) return;
    const float inv_n = sp.inv_nsites;
    const int kmx = fp.kmax[0], kmy = fp.kmax[1];
    const bool noisy = fp.noisy != 0 && a.seg_noise != nullptr;
    const float sigma0 = fp.sigma0;
    C *gb = WB + g * S::WS;
    unsigned long long target = 0;
    bool alive = true;
    float acc[11], cmp[11];   // the thread's gradient terms over the segment: compensated sums
#pragma unroll
    for (int k = 0; k < 11; ++k) acc[k] = cmp[k] = 0.f;

#pragma unroll 1
    for (int it = 0; it <= a.len && alive; ++it) {
        const int ib = a.len - it;        // the step whose part B runs (it >= 1), after its x pass
        const int ia = a.len - 1 - it;    // the step whose part A runs (it < len)
        if (it > 0) {
            // ================= row phase: the x pass of step ib =================
            target += nb;
            grid_arrive<NT>(a.gs);
            alive = grid_wait<NT>(a.gs, target, a.d_status, sp.wait_limit, &s_abort);
            if (!alive) break;
            if (npr > 0) {
                const int r0 = 2 * p0;
                // the CTA's real rows of step ib (one contiguous run), then nu's rows staged as
                // Y = conj(Z) (k2_row, ROW_ADJ) into each group's second buffer
                {
                    const float4 *__restrict__ src =
                        reinterpret_cast<const float4 *>(a.seg_real + (size_t)ib * a.rstride + (size_t)r0 * N);
                    float4 *ms4 = reinterpret_cast<float4 *>(MS);
                    const int n4 = npr * N / 2;
#pragma unroll 4
                    for (int q = t; q < n4; q += NT) ms4[q] = __ldcg(src + q);
                }
                const int ntl = (sp.hx + 3) >> 2;
                const float4 *__restrict__ nu4 = reinterpret_cast<const float4 *>(a.NU);
                for (int idx = t; idx < ntl * NG; idx += NT) {
                    const int tl = idx / NG, j = idx - tl * NG;
                    if (j >= npr) continue;
                    const float4 *p = nu4 + ((size_t)tl * N + r0 + 2 * j) * 2;
                    float4 v[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) v[q] = __ldcg(p + q);
                    C *Y = WB + j * S::WS + S::BUF;
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int k = 4 * tl + c;
                        if (k > N / 2) break;
                        const float4 va = v[c >> 1], vb = v[2 + (c >> 1)];
                        float ar = (c & 1) ? va.z : va.x, ai = (c & 1) ? va.w : va.y;
                        float br = (c & 1) ? vb.z : vb.x, bi = (c & 1) ? vb.w : vb.y;
                        if (k >= sp.hx) { ar = 0.f; ai = 0.f; br = 0.f; bi = 0.f; }
                        if (k == 0 || k == N / 2) { ai = 0.f; bi = 0.f; }   // the half spectra of real rows
                        const C lo = mk<float>(ar - bi, -ai - br), hi = mk<float>(ar + bi, ai - br);
                        Y[k] = lo;
                        if (k > 0 && k < N / 2) Y[N - k] = hi;
                    }
                }
                main_sync<NT>();
                // z' = F(Y); its last pass multiplies by p r^(p-1) (the linearised power); W = F(z'')
                if (g < npr) {
                    C *b0 = gb, *b1 = gb + S::BUF;
                    const float *ma = MS + (size_t)(2 * g) * N, *mb = ma + N;
                    C *o = fft_fwd_group<N, E, 2>(b1, b0, b1, gl, 1 + g, TW, fp.power, nullptr, nullptr, ma, mb);
                    C *o2 = fft_fwd_group<N, E, 2>(o, o == b0 ? b1 : b0, o, gl, 1 + g, TW, 0);
                    if (t == 0) s_o2 = (int)(o2 - gb);
                }
                main_sync<NT>();
                // the two rows' half spectra, stored tiled: (tile, pair j) as the 64 bytes of its rows
                const C *o2w = WB + s_o2;
                float4 *__restrict__ w4 = reinterpret_cast<float4 *>(a.W);
                for (int idx = t; idx < sp.ntiles * NG; idx += NT) {
                    const int tl = idx / NG, j = idx - tl * NG;
                    if (j >= npr) continue;
                    const C *Wj = o2w + j * S::WS;
                    float4 ab[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int k = 4 * tl + c;
                        ab[c] = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (k <= N / 2) {
                            const C wk = Wj[k], wm = Wj[(N - k) & (N - 1)];
                            ab[c] = make_float4(0.5f * (wk.x + wm.x), 0.5f * (wk.y - wm.y), 0.5f * (wk.y + wm.y),
                                                -0.5f * (wk.x - wm.x));
                        }
                    }
                    float4 *p = w4 + ((size_t)tl * N + r0 + 2 * j) * 2;
                    p[0] = make_float4(ab[0].x, ab[0].y, ab[1].x, ab[1].y);   // row a
                    p[1] = make_float4(ab[2].x, ab[2].y, ab[3].x, ab[3].y);
                    p[2] = make_float4(ab[0].z, ab[0].w, ab[1].z, ab[1].w);   // row b
                    p[3] = make_float4(ab[2].z, ab[2].w, ab[3].z, ab[3].w);
                }
            }
            target += nb;
            grid_arrive<NT>(a.gs);
            alive = grid_wait<NT>(a.gs, target, a.d_status, sp.wait_limit, &s_abort);
            if (!alive) break;
        }
        // ================= column phase: each group on its own column =================
        // part B of step ib (it >= 1): lambda = mu + F_y[w] / N on the kept modes, then the
        // Hermitian part on kx = 0, Nx/2; part A of step ia (ia >= 0): mu = g lambda, the
        // gradient terms, conj(nu) = conj(dt M mu) with F_y of the step's product, and nu
        // back along y from registers.  A thread owns the modes ky = gl + TPF m of its
        // group's column in both parts.  A CTA with at most NG / 2 columns lets its other
        // groups transform the product (part A's F_y) while the column's group runs part B
        // ("split"); otherwise the column's group runs both, part A's arithmetic on the last
        // pass of that transform.
        {
            constexpr int RES = S::NPASS % 2 == 1 ? 0 : S::BUF;   // fft_regs_smem's result in its buffers
            const bool split = ncs <= NG / 2;
            const bool lead = !split || g < NG / 2;                // the column's own group
            const int col = lead ? g : g - NG / 2;
            const int kx = 2 * u0 + col;
            const bool mine = col < ncs && kx < sp.hx;
            C *b0 = gb, *b1 = gb + S::BUF;
            C *x3 = X3 + col * N;
            const bool kxk = kx <= kmx, herm = kx == 0 || 2 * kx == sp.nx;
            C x[E];
            if (!lead && mine && ia >= 0) {
                // the step's product (column-major) transformed by this helper group
                const C *__restrict__ pr = a.seg_prod + (size_t)ia * a.cstride + (size_t)kx * N + gl;
#pragma unroll
                for (int m = 0; m < E; ++m) x[m] = __ldcg(pr + m * TPF);
                fft_regs_smem<N, E>(x, b0, b1, gl, 1 + g, TW);
            }
            C ph[E], xi[E];
            if (lead && mine) {
                if (it > 0) {
#pragma unroll
                    for (int m = 0; m < E; ++m) x[m] = __ldcg(a.W + tiled(kx, gl + m * TPF));
                    fft_regs_sink<N, E>(x, b0, b1, gl, 1 + g, TW, [&](int ky, C pv) {
                        const bool keep = kxk && abs(signed_k(ky, N)) <= kmy;
                        const C mu = x3[ky];
                        x3[ky] = keep ? mk<float>(mu.x + pv.x * inv_n, mu.y + pv.y * inv_n) : mu;
                    });
                    group_sync<TPF>(1 + g);
                    if (herm) {
                        for (int pos = gl; pos < N / 2 + 1; pos += TPF) {
                            const int ppos = (N - pos) & (N - 1);
                            const C v0 = x3[pos], v1 = x3[ppos];
                            const C h = mk<float>(0.5f * (v0.x + v1.x), 0.5f * (v0.y - v1.y));
                            x3[pos] = h;
                            x3[ppos] = mk<float>(h.x, -h.y);
                        }
                        group_sync<TPF>(1 + g);
                    }
                }
                if (ia >= 0) {
                    // the state after step ia and its noise (tiled) at the thread's modes, and
                    // (not split) the step's product, all loads in flight together
                    const C *__restrict__ pr = a.seg_prod + (size_t)ia * a.cstride + (size_t)kx * N + gl;
                    const C *__restrict__ phn = a.seg_state + (size_t)(ia + 1) * a.cstride;
                    const C *__restrict__ nzn = noisy ? a.seg_noise + (size_t)ia * a.cstride : nullptr;
#pragma unroll
                    for (int m = 0; m < E; ++m) {
                        const int ky = gl + m * TPF;
                        if (!split) x[m] = __ldcg(pr + m * TPF);
                        ph[m] = __ldcg(phn + tiled(kx, ky));
                        xi[m] = noisy ? cscale<float>(__ldcg(nzn + tiled(kx, ky)), sigma0) : mk<float>(0.f, 0.f);
                    }
                }
            }
            if (split) main_sync<NT>();   // the helpers' transforms are in place
            if (lead && mine && ia >= 0) {
                const float qx = float(kx) * sp.gx;
                const float wgt = herm ? 1.f : 2.f;
                float st[11];
#pragma unroll
                for (int k = 0; k < 11; ++k) st[k] = 0.f;
                // part A at mode ky (register m) with the product's transform pv: mu = g lambda
                // (stored), the gradient terms, conj(nu)
                auto part_a = [&](int ky, int m, C pv) {
                    const float qy = float(signed_k(ky, N)) * sp.gy;
                    const float q2 = qx * qx + qy * qy;
                    const float gg = 1.f / (1.f + sp.dt * poly5<float>(fp.O, q2));
                    const C mu = cscale<float>(x3[ky], gg);
                    x3[ky] = mu;
                    const float dtM = fp.power > 0 ? sp.dt * poly5<float>(fp.M, q2) : 0.f;
                    const float a_phi = wgt * sp.dt * (mu.x * ph[m].x + mu.y * ph[m].y);
                    const float a_P = wgt * sp.dt * (mu.x * pv.x + mu.y * pv.y);
                    float q2k = 1.f;
#pragma unroll
                    for (int k = 0; k < 5; ++k) {
                        st[k] -= q2k * a_phi;
                        st[5 + k] += q2k * a_P;
                        q2k *= q2;
                    }
                    st[10] += wgt * (mu.x * xi[m].x + mu.y * xi[m].y);
                    return mk<float>(mu.x * dtM, -mu.y * dtM);   // conj(nu)
                };
                if (split) {
                    const C *P = WB + (size_t)(col + NG / 2) * S::WS + RES;
#pragma unroll
                    for (int m = 0; m < E; ++m) x[m] = part_a(gl + m * TPF, m, P[gl + m * TPF]);
                } else {
                    fft_regs_regs_m<N, E>(x, b0, b1, gl, 1 + g, TW, part_a);
                }
                // the step's terms into the thread's compensated running sums (TwoSum)
#pragma unroll
                for (int k = 0; k < 11; ++k) {
                    const float sm = __fadd_rn(acc[k], st[k]), bp = __fsub_rn(sm, acc[k]);
                    cmp[k] = __fadd_rn(cmp[k], __fadd_rn(__fsub_rn(acc[k], __fsub_rn(sm, bp)), __fsub_rn(st[k], bp)));
                    acc[k] = sm;
                }
                // y-inverse of conj(nu); its first pass into the buffer the last pass did not read
                // (split: both are free since the barrier after part B)
                C *fr = SinkShape<N, E>::LAST_READS_B1 ? b0 : b1;
                C *__restrict__ nu = a.NU;
                fft_regs_sink<N, E>(x, fr, fr == b0 ? b1 : b0, gl, 1 + g, TW,
                                    [&](int q, C v) { nu[tiled(kx, q)] = mk<float>(v.x, -v.y); });
            }
        }
    }
    if (!alive) {
        s_abort = 1;
        return;
    }
    // the adjoint field of the segment's first step back to the tiled array
    main_sync<NT>();
    for (int i = t; i < ncs * N; i += NT) {
        const int c = i >> ilog2(N), ky = i & (N - 1), kx = 2 * u0 + c;
        if (kx < sp.hx) a.L[tiled(kx, ky)] = X3[i];
    }
    // the gradient sums: each thread's compensated sum in FP64, summed over the warp,
    // the CTA (shared memory) and the grid (one FP64 atomic per value and CTA)
#pragma unroll
    for (int k = 0; k < 11; ++k) {
        double v = (double)acc[k] + (double)cmp[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((t & 31) == 0 && v != 0.0) atomicAdd(&red[k], v);
    }
    main_sync<NT>();
    if (t < 11 && red[t] != 0.0) atomicAdd(&a.grad[t], red[t]);
    // the last CTA to finish sets the barrier words back for the next launch
    if (t == 0 && atomicAdd(&a.gs->done, 1u) == nb - 1) {
        a.gs->count = 0ull;
        a.gs->done = 0u;
    }
}

}  // namespace pss

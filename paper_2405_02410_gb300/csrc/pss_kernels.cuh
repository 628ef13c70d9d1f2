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
#pragma once

#include "pss_device.cuh"
#include "pss_internal.h"

namespace pss {

constexpr int W = kTileW;

template <typename T> __device__ __forceinline__ T poly5(const T *c, T x) {
    return (((c[4] * x + c[3]) * x + c[2]) * x + c[1]) * x + c[0];
}

template <typename T> __device__ __forceinline__ int signed_k(int k, int n) { return k < (n + 1) / 2 ? k : k - n; }

// Noise increment xi_q of one mode of the half spectrum (Eq. noise_eq over one
// step).  Each Hermitian pair is drawn once, with Philox counter word 0 = the
// smaller of the two half-spectrum indices [kz][ky][kx]; a mode that is its
// own partner is real.
template <typename T>
__device__ __forceinline__ cplx<T> noise_mode(int kx, int ky, int kz, T q2, const SysP<T> &sp,
                                              const FieldP<T> &fp, uint32_t step) {
    const uint32_t own = (uint32_t)(((long long)kz * sp.ny + ky) * sp.hx + kx);
    uint32_t canon = own;
    bool cj = false, selfc = false;
    if (kx == 0 || 2 * kx == sp.nx) {
        const int pky = (sp.ny - ky) % sp.ny, pkz = (sp.nz - kz) % sp.nz;
        const uint32_t par = (uint32_t)(((long long)pkz * sp.ny + pky) * sp.hx + kx);
        selfc = par == own;
        if (par < own) { canon = par; cj = true; }
    }
    const u32x4 r = philox4x32_10(u32x4{canon, step, (uint32_t)fp.field_id, 0u}, sp.seed_lo, sp.seed_hi);
    T n1, n2;
    box_muller(uniform24<T>(r.x), uniform24<T>(r.y), n1, n2);
    T q2p = T(1);
    for (int p = 0; p < fp.noise_pow; ++p) q2p *= q2;
    const T amp = sqrt(fp.amp2 * q2p);
    if (selfc) return mk<T>(T(1.4142135623730951) * amp * n1, T(0));
    return mk<T>(amp * n1, cj ? -amp * n2 : amp * n2);
}

// ---------------------------------------------------------------------------
// k_col: FFTs along the slowest axis (N = n_inner points), fused with the
// update.  CTA = tiles_per_cta tiles x NP pencils x kTileW columns; in 3D the
// two pencils are ky and -ky so that the Hermitian pair of every kx = 0 mode
// sits in the same CTA.
// ---------------------------------------------------------------------------
template <typename T, int N>
__global__ void __launch_bounds__(256) k_col(const ColArgs<T> a) {
    using C = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *sbuf = reinterpret_cast<C *>(smem_raw);
    constexpr int E = FftShape<N>::E, TPF = FftShape<N>::TPF;
    const SysP<T> &sp = a.sp;
    const int fld = blockIdx.z;
    const FieldP<T> &fp = a.fp[fld];
    const int NP = sp.dim == 3 ? 2 : 1;
    const int F = a.tiles_per_cta * W * NP;
    const int t = threadIdx.x;
    const int f = t % F, lane = t / F;
    const int c = f % W, pp = (f / W) % NP, tl = f / (W * NP);
    const int tile = blockIdx.x * a.tiles_per_cta + tl;
    const int op = blockIdx.y;
    const int o = pp == 0 ? op : (sp.n_outer - op) % sp.n_outer;
    const bool tile_ok = tile < a.n_tiles;
    const bool writer = tile_ok && !(pp == 1 && o == op);
    const int kx = tile * W + c;
    const size_t base = ((size_t)(tile * sp.n_outer + o) * N) * W + c;
    const C *__restrict__ tw = a.tw;
    const int mode = a.mode;

    C v[E];
    const C *src = (mode == COL_STEP || mode == COL_FWD) ? a.in[fld] : a.state[fld];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = tile_ok ? src[base + (size_t)(lane + TPF * e) * W] : mk<T>(0, 0);

    if (mode == COL_STEP || mode == COL_FWD) {
        fft<T, N, -1>(v, lane, sbuf, F, f, tw);
        const uint32_t step = (uint32_t)(*a.d_step);
        C *__restrict__ st = a.state[fld];
        bool bad = false;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int pos = lane + TPF * e;
            const int ky = sp.dim == 3 ? o : (sp.dim == 2 ? pos : 0);
            const int kz = sp.dim == 3 ? pos : 0;
            C phi;
            if (mode == COL_FWD) {
                phi = v[e];
            } else {
                phi = tile_ok ? st[base + (size_t)pos * W] : mk<T>(0, 0);
                const T qx = T(kx) * sp.gx, qy = T(signed_k<T>(ky, sp.ny)) * sp.gy,
                        qz = T(signed_k<T>(kz, sp.nz)) * sp.gz;
                const T q2 = qx * qx + qy * qy + qz * qz;
                C num = phi;
                if (fp.power > 0) {
                    const T dtM = sp.dt * poly5<T>(fp.M, q2);
                    num = mk<T>(num.x + dtM * v[e].x, num.y + dtM * v[e].y);
                }
                if (fp.noisy) num = cadd<T>(num, noise_mode<T>(kx, ky, kz, q2, sp, fp, step));
                const T den = T(1) + sp.dt * poly5<T>(fp.O, q2);
                phi = mk<T>(num.x / den, num.y / den);
                bad |= !(isfinite(phi.x) && isfinite(phi.y));
            }
            if (kx >= sp.hx) phi = mk<T>(0, 0);
            v[e] = phi;
        }
        // Hermitian part on the kx = 0 and kx = Nx/2 planes (the field is real)
        const int first = blockIdx.x * a.tiles_per_cta * W, last = first + a.tiles_per_cta * W;
        const bool proj = first == 0 || (first <= sp.nx / 2 && sp.nx / 2 < last);
        if (proj) {
            __syncthreads();
#pragma unroll
            for (int e = 0; e < E; ++e) sbuf[spad(lane + TPF * e) * F + f] = v[e];
            __syncthreads();
            const int fp2 = NP == 2 ? (pp == 0 ? f + W : f - W) : f;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int pos = lane + TPF * e;
                const int ppos = (N - pos) & (N - 1);
                const C q = sbuf[spad(ppos) * F + fp2];
                if (kx == 0 || 2 * kx == sp.nx) v[e] = mk<T>(T(0.5) * (v[e].x + q.x), T(0.5) * (v[e].y - q.y));
            }
            __syncthreads();
        }
        if (writer) {
#pragma unroll
            for (int e = 0; e < E; ++e) st[base + (size_t)(lane + TPF * e) * W] = v[e];
        }
        if (bad && a.d_status) atomicOr(a.d_status, 1);
        if (mode == COL_FWD) return;
    }

    // ---- inverse along this axis: de-alias (not for COL_INV_FULL), scale by 1/N_sites
    const bool full = mode == COL_INV_FULL;
    if (!full) {
        // CTA-uniform early exit when no column or pencil of the CTA is kept
        const int first_kx = blockIdx.x * a.tiles_per_cta * W;
        const int ky0 = op;
        const bool ky_kept = sp.dim != 3 || abs(signed_k<T>(ky0, sp.ny)) <= fp.kmax[1];
        if (first_kx > fp.kmax[0] || !ky_kept) return;
    }
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int pos = lane + TPF * e;
        bool keep = kx < sp.hx;
        if (!full) {
            const int ky = sp.dim == 3 ? o : (sp.dim == 2 ? pos : 0);
            const int kz = sp.dim == 3 ? pos : 0;
            keep = keep && kx <= fp.kmax[0] && abs(signed_k<T>(ky, sp.ny)) <= fp.kmax[1] &&
                   abs(signed_k<T>(kz, sp.nz)) <= fp.kmax[2];
        }
        v[e] = keep ? cscale<T>(v[e], sp.inv_nsites) : mk<T>(0, 0);
    }
    fft<T, N, +1>(v, lane, sbuf, F, f, tw);
    if (writer && (full || tile * W <= fp.kmax[0])) {
        C *__restrict__ dst = a.out[fld];
#pragma unroll
        for (int e = 0; e < E; ++e) dst[base + (size_t)(lane + TPF * e) * W] = v[e];
    }
}

// ---------------------------------------------------------------------------
// k_row: transforms along x (N = nx) for G pairs of rows per CTA.  Two real
// rows a, b ride on one complex FFT z = a + i b: C2R builds
// Z_k = A_k + i B_k from the two half spectra, and R2C splits the transform W
// of z by A_k = (W_k + conj W_{N-k}) / 2, B_k = (W_k - conj W_{N-k}) / (2i).
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

template <typename T, int N>
__global__ void __launch_bounds__(256) k_row(const RowArgs<T> a) {
    using C = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *S = reinterpret_cast<C *>(smem_raw);
    T *Sr = reinterpret_cast<T *>(smem_raw);
    constexpr int E = FftShape<N>::E, TPF = FftShape<N>::TPF;
    const SysP<T> &sp = a.sp;
    const int G = a.G, G2 = 2 * a.G;
    const int fld = blockIdx.y;
    const int t = threadIdx.x, nthr = blockDim.x;
    const int g = t % G, lane = t / G;
    const int r0 = blockIdx.x * G2;
    const int rows = sp.rows;
    const C *__restrict__ tw = a.tw;
    const int mode = a.mode;
    C v[E];

    if (mode == ROW_R2C) {
        const T *__restrict__ src = a.real_in[fld];
        for (int L = t; L < G2 * N; L += nthr) {
            const int x = L % N, rl = L / N, row = r0 + rl;
            Sr[x * G2 + rl] = row < rows ? src[real_row_offset(sp, row) + x] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int k = lane + TPF * e;
            v[e] = mk<T>(Sr[k * G2 + g], Sr[k * G2 + G + g]);
        }
        __syncthreads();
    } else {
        const C *__restrict__ src = a.in[fld];
        const int kxc = a.kx_cols[fld];
        const int ntl = (kxc + W - 1) / W;
        for (int L = t; L < ntl * G2 * W; L += nthr) {
            const int cc = L % W, rl = (L / W) % G2, tl = L / (W * G2);
            const int kx = tl * W + cc, row = r0 + rl;
            if (kx < kxc) S[kx * G2 + rl] = row < rows ? src[((size_t)tl * rows + row) * W + cc] : mk<T>(0, 0);
        }
        __syncthreads();
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int k = lane + TPF * e;
            const int kk = k <= N / 2 ? k : N - k;
            C xa = kk < kxc ? S[kk * G2 + g] : mk<T>(0, 0);
            C xb = kk < kxc ? S[kk * G2 + G + g] : mk<T>(0, 0);
            if (k > N / 2) { xa.y = -xa.y; xb.y = -xb.y; }
            if (k == 0 || 2 * k == N) { xa.y = T(0); xb.y = T(0); }
            v[e] = mk<T>(xa.x - xb.y, xa.y + xb.x);
        }
        __syncthreads();
        fft<T, N, +1>(v, lane, S, G, g, tw);
        if (mode == ROW_C2R) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int x = lane + TPF * e;
                Sr[x * G2 + g] = v[e].x;
                Sr[x * G2 + G + g] = v[e].y;
            }
            __syncthreads();
            T *__restrict__ dst = a.real_out[fld];
            for (int L = t; L < G2 * N; L += nthr) {
                const int x = L % N, rl = L / N, row = r0 + rl;
                if (row < rows) dst[real_row_offset(sp, row) + x] = Sr[x * G2 + rl];
            }
            return;
        }
        // real-space product of the de-aliased field
        const int p = a.power[fld];
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = mk<T>(ipow<T>(v[e].x, p), ipow<T>(v[e].y, p));
    }
    fft<T, N, -1>(v, lane, S, G, g, tw);
#pragma unroll
    for (int e = 0; e < E; ++e) S[spad(lane + TPF * e) * G + g] = v[e];
    __syncthreads();
    C *__restrict__ dst = a.out[fld];
    const int ntl = sp.ntiles;
    for (int L = t; L < ntl * G2 * W; L += nthr) {
        const int cc = L % W, rl = (L / W) % G2, tl = L / (W * G2);
        const int kx = tl * W + cc, row = r0 + rl;
        if (row >= rows) continue;
        C val = mk<T>(0, 0);
        if (kx <= N / 2) {
            const int gg = rl % G;
            const C wk = S[spad(kx) * G + gg];
            const C wm = S[spad((N - kx) & (N - 1)) * G + gg];
            val = rl < G ? mk<T>(T(0.5) * (wk.x + wm.x), T(0.5) * (wk.y - wm.y))
                         : mk<T>(T(0.5) * (wk.y + wm.y), T(-0.5) * (wk.x - wm.x));
        }
        dst[((size_t)tl * rows + row) * W + cc] = val;
    }
    if (a.inc_step && blockIdx.x == 0 && blockIdx.y == 0 && t == 0) *a.d_step += 1;
}

// ---------------------------------------------------------------------------
// k_mid: FFTs along y in 3D (N = ny points) for one tile and PZ z-planes.
// ---------------------------------------------------------------------------
template <typename T, int N>
__global__ void __launch_bounds__(256) k_mid(const MidArgs<T> a) {
    using C = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *sbuf = reinterpret_cast<C *>(smem_raw);
    constexpr int E = FftShape<N>::E, TPF = FftShape<N>::TPF;
    const SysP<T> &sp = a.sp;
    const int fld = blockIdx.z;
    const int F = a.PZ * W;
    const int t = threadIdx.x;
    const int f = t % F, lane = t / F;
    const int c = f % W, pz = f / W;
    const int tile = blockIdx.x;
    const int pos = blockIdx.y * a.PZ + pz;
    const int nz = sp.nz;
    const size_t base = ((size_t)tile * N * nz + pos) * W + c;   // + o * nz * W
    const C *__restrict__ src = a.in[fld];
    const bool masked_in = a.mode == MID_INV_MASK;
    const int kmy = a.kmax_y[fld];
    C v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int o = lane + TPF * e;
        const bool ld = !masked_in || abs(signed_k<T>(o, N)) <= kmy;
        v[e] = ld ? src[base + (size_t)o * nz * W] : mk<T>(0, 0);
    }
    if (a.mode == MID_FWD) fft<T, N, -1>(v, lane, sbuf, F, f, a.tw);
    else fft<T, N, +1>(v, lane, sbuf, F, f, a.tw);
    C *__restrict__ dst = a.out[fld];
#pragma unroll
    for (int e = 0; e < E; ++e) dst[base + (size_t)(lane + TPF * e) * nz * W] = v[e];
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
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int kx = (int)(i % sp.hx);
        const long long r2 = i / sp.hx;
        const int ky = (int)(r2 % sp.ny), kz = (int)(r2 / sp.ny);
        const int ks[3] = {kx, signed_k<T>(ky, sp.ny), signed_k<T>(kz, sp.nz)};
        double s2 = 0.0, qq = 0.0;
        for (int j = 0; j < 3; ++j) {
            if (Ns[j] == 1) continue;
            const double num = __dmul_rn(__dmul_rn(__dmul_rn(2.0, (double)nbins), (double)ks[j]), dx0);
            const double tj = __ddiv_rn(num, __dmul_rn((double)Ns[j], dxs[j]));
            s2 = __dadd_rn(s2, __dmul_rn(tj, tj));
            const double qj = 6.283185307179586 * ks[j] / (Ns[j] * dxs[j]);
            qq += qj * qj;
        }
        if (s2 == 0.0) continue;
        const double s = __dsqrt_rn(s2);
        if (s > (double)nbins) continue;
        const int b = (int)ceil(s) - 1;
        const int row = sp.dim == 3 ? ky * sp.nz + kz : ky;
        const cplx<T> z = tiles[((size_t)(kx / W) * sp.rows + row) * W + kx % W];
        const double S = ((double)z.x * z.x + (double)z.y * z.y) * inv_ns;
        const double wgt = (kx == 0 || 2 * kx == sp.nx) ? 1.0 : 2.0;
        atomicAdd(&sacc[b], wgt * S);
        atomicAdd(&sacc[nbins + b], wgt);
        atomicAdd(&sacc[2 * nbins], wgt * S);
        atomicAdd(&sacc[2 * nbins + 1], wgt * sqrt(qq) * S);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 2 * nbins + 2; i += blockDim.x)
        if (sacc[i] != 0.0) atomicAdd(&acc[i], sacc[i]);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <typename T, int N> cudaError_t launch_col_n(const ColArgs<T> &a, int nf, int gx, int gy, cudaStream_t st) {
    const int NP = a.sp.dim == 3 ? 2 : 1;
    const int F = a.tiles_per_cta * W * NP;
    const int threads = F * FftShape<N>::TPF;
    const size_t smem = sizeof(cplx<T>) * (size_t)fft_smem_elems(N, F);
    if (threads > 256) return cudaErrorInvalidConfiguration;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_col<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_col<T, N><<<dim3(gx, gy, nf), threads, smem, st>>>(a);
    return cudaGetLastError();
}

template <typename T> cudaError_t launch_col(const ColArgs<T> &a, int nf, int gx, int gy, cudaStream_t st) {
    switch (a.sp.n_inner) {
        case 1: return launch_col_n<T, 1>(a, nf, gx, gy, st);
        case 4: return launch_col_n<T, 4>(a, nf, gx, gy, st);
        case 8: return launch_col_n<T, 8>(a, nf, gx, gy, st);
        case 16: return launch_col_n<T, 16>(a, nf, gx, gy, st);
        case 32: return launch_col_n<T, 32>(a, nf, gx, gy, st);
        case 64: return launch_col_n<T, 64>(a, nf, gx, gy, st);
        case 128: return launch_col_n<T, 128>(a, nf, gx, gy, st);
        case 256: return launch_col_n<T, 256>(a, nf, gx, gy, st);
        case 512: return launch_col_n<T, 512>(a, nf, gx, gy, st);
        case 1024: return launch_col_n<T, 1024>(a, nf, gx, gy, st);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T, int N> cudaError_t launch_row_n(const RowArgs<T> &a, int nf, cudaStream_t st) {
    const int G = a.G;
    const int threads = G * FftShape<N>::TPF;
    size_t elems = (size_t)fft_smem_elems(N, G);
    elems = elems > (size_t)(N / 2 + 1) * 2 * G ? elems : (size_t)(N / 2 + 1) * 2 * G;
    elems = elems > (size_t)N * G ? elems : (size_t)N * G;   // 2G rows of N reals
    const size_t smem = sizeof(cplx<T>) * elems;
    if (threads > 256) return cudaErrorInvalidConfiguration;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_row<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int grid = (a.sp.rows + 2 * G - 1) / (2 * G);
    k_row<T, N><<<dim3(grid, nf), threads, smem, st>>>(a);
    return cudaGetLastError();
}

template <typename T> cudaError_t launch_row(const RowArgs<T> &a, int nf, cudaStream_t st) {
    switch (a.sp.nx) {
        case 4: return launch_row_n<T, 4>(a, nf, st);
        case 8: return launch_row_n<T, 8>(a, nf, st);
        case 16: return launch_row_n<T, 16>(a, nf, st);
        case 32: return launch_row_n<T, 32>(a, nf, st);
        case 64: return launch_row_n<T, 64>(a, nf, st);
        case 128: return launch_row_n<T, 128>(a, nf, st);
        case 256: return launch_row_n<T, 256>(a, nf, st);
        case 512: return launch_row_n<T, 512>(a, nf, st);
        case 1024: return launch_row_n<T, 1024>(a, nf, st);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T, int N> cudaError_t launch_mid_n(const MidArgs<T> &a, int nf, int n_tiles, cudaStream_t st) {
    const int F = a.PZ * W;
    const int threads = F * FftShape<N>::TPF;
    const size_t smem = sizeof(cplx<T>) * (size_t)fft_smem_elems(N, F);
    if (threads > 256) return cudaErrorInvalidConfiguration;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_mid<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_mid<T, N><<<dim3(n_tiles, a.sp.nz / a.PZ, nf), threads, smem, st>>>(a);
    return cudaGetLastError();
}

template <typename T> cudaError_t launch_mid(const MidArgs<T> &a, int nf, int n_tiles, cudaStream_t st) {
    switch (a.sp.ny) {
        case 4: return launch_mid_n<T, 4>(a, nf, n_tiles, st);
        case 8: return launch_mid_n<T, 8>(a, nf, n_tiles, st);
        case 16: return launch_mid_n<T, 16>(a, nf, n_tiles, st);
        case 32: return launch_mid_n<T, 32>(a, nf, n_tiles, st);
        case 64: return launch_mid_n<T, 64>(a, nf, n_tiles, st);
        case 128: return launch_mid_n<T, 128>(a, nf, n_tiles, st);
        case 256: return launch_mid_n<T, 256>(a, nf, n_tiles, st);
        case 512: return launch_mid_n<T, 512>(a, nf, n_tiles, st);
        case 1024: return launch_mid_n<T, 1024>(a, nf, n_tiles, st);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t launch_init_uniform(T *real, long long nsites, double lo, double hi, uint32_t s0, uint32_t s1,
                                int field_id, cudaStream_t st) {
    const int threads = 256;
    long long blocks = (nsites + threads - 1) / threads;
    if (blocks > 65535) blocks = 65535;
    k_init_uniform<T><<<(int)blocks, threads, 0, st>>>(real, nsites, T(lo), T(hi), s0, s1, field_id);
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
    k_tiles_half<T><<<(int)blocks, 256, 0, st>>>(sp, const_cast<cplx<T> *>(tiles), const_cast<cplx<T> *>(half), 0);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_structure_factor(const SysP<T> &sp, const double dx[3], const cplx<T> *tiles, int nbins,
                                    double *acc, cudaStream_t st) {
    const long long n = (long long)sp.nz * sp.ny * sp.hx;
    long long blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    const size_t smem = sizeof(double) * (size_t)(2 * nbins + 2);
    k_structure_factor<T><<<(int)blocks, 256, smem, st>>>(sp, dx[0], dx[1], dx[2], tiles, nbins, acc);
    return cudaGetLastError();
}

#define PSS_INSTANTIATE(T)                                                                                   \
    template cudaError_t launch_col<T>(const ColArgs<T> &, int, int, int, cudaStream_t);                     \
    template cudaError_t launch_row<T>(const RowArgs<T> &, int, cudaStream_t);                               \
    template cudaError_t launch_mid<T>(const MidArgs<T> &, int, int, cudaStream_t);                          \
    template cudaError_t launch_init_uniform<T>(T *, long long, double, double, uint32_t, uint32_t, int,     \
                                                cudaStream_t);                                               \
    template cudaError_t launch_tiles_to_half<T>(const SysP<T> &, const cplx<T> *, cplx<T> *, cudaStream_t); \
    template cudaError_t launch_half_to_tiles<T>(const SysP<T> &, const cplx<T> *, cplx<T> *, cudaStream_t); \
    template cudaError_t launch_structure_factor<T>(const SysP<T> &, const double *, const cplx<T> *, int,   \
                                                    double *, cudaStream_t);

}  // namespace pss

// pss_internal.h -- types shared by the host side of libpss and its kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pss {

// complex numbers: float2 / double2 (x = real part, y = imaginary part)
template <typename T> struct CplxOf;
template <> struct CplxOf<float> { using type = float2; };
template <> struct CplxOf<double> { using type = double2; };
template <typename T> using cplx = typename CplxOf<T>::type;

// Twiddle factors: the host builds, in FP64, one table per transform length
// n = 2, 4, ..., kMaxFftN and radix cap emax (8, 16 or 32).  A length-n FFT runs
// radix-E passes (E = min(n, emax)) and a last pass of radix n / P (<= E).
// The pass that follows P > 1 points already transformed, of radix
// R = min(E, n / P), needs exp(-2 pi i r k / (P R)) for 1 <= r < R, k < P,
// which the table holds at entry (P - E) + (r - 1) P + k: n - E entries in
// all.  The table of (n, emax) starts at entry twiddle_offset(n, emax)
// (16-byte aligned, room for n entries), so kernels stage it with one bulk
// copy.
constexpr int kMaxFftN = 1024;
__host__ __device__ constexpr int twiddle_offset(int n, int emax) {
    return (emax == 32 ? 4 * kMaxFftN : emax == 16 ? 2 * kMaxFftN : 0) + n;
}
constexpr int kTwiddleEntries = 6 * kMaxFftN;

constexpr int kTileW = 4;       // kx columns per tile of every spectral array
constexpr int kMaxFields = 4;
constexpr int kPolyTerms = 5;   // operators are polynomials of degree <= 4 in q^2

// Spectral arrays are stored as [tile][row][kTileW] complex values, where
// tile = kx / kTileW over the Nx/2+1 half-spectrum columns (the last tile
// padded with zero columns) and row = o * n_inner + pos:
//   3D: o = ky (or y), pos = kz (or z);  2D: o = 0, pos = ky (or y);  1D: one row.
// A tile of one row range is contiguous, so the y/z passes read whole
// pencils of kTileW columns with unit stride and the x pass reads
// kTileW-wide segments of many rows at once.

// Parameters of one (instance, field) slot.  Slots are numbered
// slot = instance * n_fields + field; every array of a system holds its slots
// back to back, slot_stride elements apart.
template <typename T> struct FieldP {
    T O[kPolyTerms];      // implicit operator O(q) = sum O[p] (q^2)^p  (L~ = -O)
    T M[kPolyTerms];      // explicit operator M(q) applied to the product term
    T sigma0;             // sqrt(N_sites D dt / dV): noise std per component is sigma0 |q|^noise_pow
    int noise_pow;        // D~ = D (q^2)^noise_pow
    int noisy;
    int power;            // product (phi^d)^power; 0 = no explicit term
    int spectral;         // the column kernel gets the product transformed along every axis (product terms)
    int kmax[3];          // largest kept |k| per axis of the de-alias mask
    int kx_cols;          // kept half-spectrum columns (kmax[0] + 1, at most Nx/2 + 1)
    int field_id;         // Philox counter word 2
    uint32_t seed_lo, seed_hi;   // Philox key of the slot's instance
};

template <typename T> struct SysP {
    int dim, nx, ny, nz, hx;
    int hxe;              // hx rounded up to even (row width of the noise counter)
    int ntiles, rows;     // rows = ny * nz
    int n_outer, n_inner;
    T gx, gy, gz;         // 2 pi / (N dx) per axis (0 for unused axes)
    T dt, inv_nsites;
    int pdl;              // launch with programmatic stream serialisation
    // bounded-wait check (tuning key "test_timeout"): polls before a wait of
    // the generic column kernel gives up (0: the default limit), and bytes
    // its first CTA's mbarrier expects beyond what its copies deliver
    int wait_limit;
    uint32_t tx_extra;
};

enum ColMode {
    COL_STEP = 0, COL_FWD = 1, COL_INV_MASK = 2, COL_INV_FULL = 3,
    COL_ADJ_A = 4,   // adjoint: mu = g lambda, coefficient gradients, inverse of nu = dt M mu (all columns)
    COL_ADJ_B = 5,   // adjoint: lambda = mu + m F[w] / N
    COL_ADJ_BA = 6   // adjoint: COL_ADJ_B of one step, then COL_ADJ_A of the step before it
};
enum RowMode {
    ROW_FUSED = 0,      // C2R of the kept columns, power p, R2C (real_out: also store the real field)
    ROW_R2C = 1, ROW_C2R = 2,
    ROW_C2R_KEPT = 3,   // C2R of the kept columns only
    ROW_ADJ = 4         // adjoint: C2R of all columns (s), times p r^(p-1) with r from real_in, R2C
};
enum MidMode { MID_INV_MASK = 0, MID_INV_FULL = 1, MID_FWD = 2 };

// Arrays: slot s of an array starts at base + s * slot_stride (complex
// elements; real arrays: s * real_stride reals).  A launch covers slots
// slot0 .. slot0 + gridDim.z - 1.
template <typename T> struct ColArgs {
    SysP<T> sp;
    const FieldP<T> *fps;
    const cplx<T> *in;
    cplx<T> *out;
    cplx<T> *state;
    cplx<T> *state_out;   // where the updated state goes (nullptr: back to state)
    size_t slot_stride;
    int slot0;
    const cplx<T> *tw;
    long long *d_step;    // step counter (k2_col advances it)
    int *d_status;
    int mode, tiles_per_cta, n_tiles;
    int E;                // FFT radix cap (8 or 16), chosen by the host
    int F;                // FFTs per CTA = tiles_per_cta * kTileW * (2 in 3D, else 1); a power of two
    // adjoint (COL_ADJ_A): the forward state after the step, its noise step, and
    // the FP64 gradient sums [slot][11] (dO_0..4, dM_0..4, sum Re(conj(mu) xi))
    const cplx<T> *aux;
    long long adj_step;
    const long long *d_adj_base;   // if set, the noise step is adj_step + *d_adj_base
    double *grad;
    int aux_warps;        // k2_col: warps that join the update beside the FFT warps
    int in_colmajor;      // k_col: `in` holds each tile's columns one after another ([c][pos]), as the
                          // FP32 2D path writes its product (the adjoint reads it)
    const cplx<T> *noise; // k2_col: unit-amplitude noise of this step (tiled like the state)
    // COL_ADJ_BA: the product of the earlier step (the A part's input; `in` is the
    // B part's), column-major like `in_colmajor` says
    const cplx<T> *in2;
    int in2_colmajor;
    // COL_INV_MASK of a product-term factor: the kept modes times
    // op(q) = (i q_op_deriv if op_deriv >= 0) (-q^2)^op_lap (op_on = 1)
    int op_on, op_deriv, op_lap;
};

template <typename T> struct RowArgs {
    SysP<T> sp;
    const FieldP<T> *fps;
    const cplx<T> *in;
    cplx<T> *out;
    const T *real_in;
    T *real_out;
    size_t slot_stride, real_stride;
    int slot0;
    const cplx<T> *tw;
    long long *d_step;
    int *d_status;
    int mode, G, inc_step;
    int E;                // FFT radix cap (8 or 16)
    int kx_cols_max;      // largest kept half-spectrum column count over the launch's slots
    cplx<T> *noise;       // k2_row: where the unit-amplitude noise of step *d_step goes (null: none)
    int noise_warps;      // k2_row: warps that draw it beside the transform warps
    int noise_ctas;       // k2_row: extra CTAs (past the row CTAs) that only draw noise
    int noise_share;      // k2_row: the pairs those CTAs draw, out of 64 (the row CTAs draw the rest)
    // ROW_C2R_KEPT of a product-term factor (fac_acc set): instead of storing
    // the real rows r, fold r^fac_power into the running product fac_tp (the
    // first factor starts it) and, at the term's last factor, add the
    // product to fac_acc (the first term of a sum starts it)
    T *fac_acc, *fac_tp;
    int fac_power, fac_first_factor, fac_last_factor, fac_first_term;
};

template <typename T> struct MidArgs {
    SysP<T> sp;
    const FieldP<T> *fps;
    const cplx<T> *in;
    cplx<T> *out;
    size_t slot_stride;
    int slot0;
    const cplx<T> *tw;
    long long *d_step;
    int *d_status;
    int mode, PZ, inc_step;
    int E;                // FFT radix cap (8 or 16)
};

// Launch configuration chosen by the host.
struct ColCfg { int tiles_per_cta; };
struct RowCfg { int G; };
struct MidCfg { int PZ; };

// Launchers of the step kernels, one instantiation per precision and FFT
// radix cap EMAX (pss_kern_{f32,f64}.cu: 8, pss_kern_{f32,f64}_r16.cu: 16).
template <typename T, int EMAX>
cudaError_t launch_col_e(const ColArgs<T> &a, int nslots, int grid_x, int grid_y, cudaStream_t st);
template <typename T, int EMAX> cudaError_t launch_row_e(const RowArgs<T> &a, int nslots, cudaStream_t st);
template <typename T, int EMAX> cudaError_t launch_mid_e(const MidArgs<T> &a, int nslots, int n_tiles, cudaStream_t st);
// dynamic shared memory of one column-kernel CTA (0: side not supported)
template <typename T, int EMAX> size_t col_smem_bytes_e(int n_inner, int F, int mode);
template <typename T> inline size_t col_smem_bytes(int n_inner, int F, int E, int mode) {
    return E == 16 ? col_smem_bytes_e<T, 16>(n_inner, F, mode) : col_smem_bytes_e<T, 8>(n_inner, F, mode);
}
template <typename T>
inline cudaError_t launch_col(const ColArgs<T> &a, int nslots, int grid_x, int grid_y, cudaStream_t st) {
    return a.E == 16 ? launch_col_e<T, 16>(a, nslots, grid_x, grid_y, st) : launch_col_e<T, 8>(a, nslots, grid_x, grid_y, st);
}
template <typename T> inline cudaError_t launch_row(const RowArgs<T> &a, int nslots, cudaStream_t st) {
    return a.E == 16 ? launch_row_e<T, 16>(a, nslots, st) : launch_row_e<T, 8>(a, nslots, st);
}
template <typename T> inline cudaError_t launch_mid(const MidArgs<T> &a, int nslots, int n_tiles, cudaStream_t st) {
    return a.E == 16 ? launch_mid_e<T, 16>(a, nslots, n_tiles, st) : launch_mid_e<T, 8>(a, nslots, n_tiles, st);
}
// The FP32 path with one FFT group per transform (sides 256, 512 or 1024):
// k2_col over `ntiles` tiles of every slot, k2_row over all row pairs.  In
// the 2D step the work arrays they exchange are column-major ([kx][y] per
// slot); with tiled = true k2_row reads and writes the tiled arrays of the
// generic kernels (the x pass of the 3D step).
cudaError_t launch_col2(const ColArgs<float> &a, int nslots, int ntiles, cudaStream_t st);
cudaError_t launch_row2(const RowArgs<float> &a, int nslots, cudaStream_t st, bool tiled);
// the adjoint's column part (COL_ADJ_A / _B / _BA) of an FP32 2D system with
// 256..1024-point columns on FFT groups, one column pair per CTA
cudaError_t launch_col2_adj(const ColArgs<float> &a, int nslots, cudaStream_t st);
// The persistent FP32 2D step (k2p_step: square sides of 256, 512 or 1024
// points, one field, one instance): grid-barrier words of one system
// (16 bytes, zero-initialised) and the launch arguments.  Barrier i of a
// launch (0-based) completes when gs->count reaches (i + 1) gridDim.x; the
// last CTA to finish a launch sets count back to 0.
struct GridSync {
    unsigned long long count;   // CTA arrivals at the launch's grid barriers so far
    unsigned int abort;         // a CTA gave up waiting: the others leave too
    unsigned int done;          // CTAs finished (the last one resets count and done)
};
struct P2Args {
    SysP<float> sp;
    const FieldP<float> *fps;   // the field's parameters (one slot)
    float2 *state;              // tiled [tile][ny][4]
    float2 *P;                  // x-transformed product, column-major [kx][ny]
    float2 *T1;                 // conjugated y-inverse of the kept columns, column-major [kx][ny]
    float2 *T1a;                // KPZ (mode 1): the same of i q_y times the field
    float2 *xi;                 // unit-amplitude noise of the next step, tiled: read at the start, written at the end
    const float2 *tw;
    long long *d_step;
    int *d_status;
    GridSync *gs;
    int nsteps;
    int prologue;               // P does not hold the product of the state yet: compute it first
    // segment mode (the adjoint's recomputed segments; seg_state != nullptr): the
    // state of step 0 is read from seg_state, and the states of steps 1..nsteps
    // (tiled), the products of steps 0..nsteps (column-major) and their
    // de-aliased real fields ([ny][nx]) are written at seg_state + i seg_cstride,
    // seg_prod + i seg_cstride, seg_real + i seg_rstride; P, xi and the state
    // write-back at the end are not used
    float2 *seg_state, *seg_prod;
    float *seg_real;
    size_t seg_cstride, seg_rstride;
    float2 *seg_noise;          // segment mode: the unit noise of steps 0..nsteps-1 (tiled), if not null
};
// n steps in one cooperative launch of nblocks CTAs (E: FFT pass radix, 8 or 16;
// mode 0: a power of the field, 1: the KPZ gradient square)
cudaError_t launch_p2(const P2Args &a, int n, int E, int nblocks, int mode, cudaStream_t st);
cudaError_t launch_p2_kpz(const P2Args &a, int n, int E, int nblocks, cudaStream_t st);
// The backward pass of one recomputed segment of the FP32 2D adjoint (k2p_adj)
struct P2AdjArgs {
    SysP<float> sp;
    const FieldP<float> *fps;   // the field's parameters (one slot)
    const float2 *tw;
    float2 *L;                  // adjoint field, tiled: of the segment's last step on entry, of its first on exit
    float2 *NU;                 // work array, tiled: nu transformed back along y
    float2 *W;                  // work array, tiled: the x pass's result
    const float2 *seg_state;    // states after steps 0..len, tiled, cstride apart
    const float2 *seg_prod;     // products of steps 0..len-1, column-major, cstride apart
    const float *seg_real;      // de-aliased real fields of steps 0..len-1 ([ny][nx]), rstride apart
    const float2 *seg_noise;    // unit noise of steps 0..len-1, tiled, cstride apart (noisy fields)
    size_t cstride, rstride;
    double *grad;               // 11 gradient sums, added to
    int *d_status;
    GridSync *gs;
    int len;                    // steps of the segment (>= 1)
};
cudaError_t launch_p2_adj(const P2AdjArgs &a, int n, int E, int nblocks, cudaStream_t st);
template <typename T> cudaError_t launch_init_uniform(T *real, long long nsites, double lo, double hi,
                                                      uint64_t seed, int field_id, cudaStream_t st);
// product terms with several operators: Q = (first ? 0 : Q) + M(q) Pt over one
// slot (m[0..4] the coefficients of M in q^2)
template <typename T>
cudaError_t launch_combine(const SysP<T> &sp, cplx<T> *Q, const cplx<T> *Pt, const double *m, int first,
                           cudaStream_t st);
template <typename T> cudaError_t launch_frame(T *real, int nx, long long rows, int width, double lo, double hi,
                                               cudaStream_t st);
template <typename T> cudaError_t launch_tiles_to_half(const SysP<T> &sp, const cplx<T> *tiles,
                                                       cplx<T> *half, cudaStream_t st);
template <typename T> cudaError_t launch_half_to_tiles(const SysP<T> &sp, const cplx<T> *half,
                                                       cplx<T> *tiles, cudaStream_t st);
template <typename T> cudaError_t launch_segment_begin(cplx<T> *dst, const cplx<T> *ck, size_t slot_elems,
                                                       const long long *d_seg, long long step_base, long long K,
                                                       long long *d_step, long long *d_adj_base, cudaStream_t st);
cudaError_t launch_set_i64(long long *dst, long long value, cudaStream_t st);
template <typename T> cudaError_t launch_structure_factor(const SysP<T> &sp, const double dx[3],
                                                          const cplx<T> *tiles, int nbins,
                                                          double *acc /* 2*nbins + 2 */, cudaStream_t st);

// FFT shape helpers visible to the host
__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n >> 1); }
// Values per thread and pass of a length-n FFT (the radix of its main
// passes) when a kernel runs its FFTs with at most emax (8 or 16) values per
// thread: radix 16 means fewer passes, radix 8 twice the threads per FFT.
__host__ __device__ constexpr int fft_E(int n, int emax) { return n < emax ? n : emax; }
__host__ __device__ constexpr int fft_TPF(int n, int emax) { return n / fft_E(n, emax); }
// threads of a column-kernel CTA with F FFTs: two per FFT lane where that
// stays within 512 (the element-wise phases use them all), at least a warp
__host__ __device__ constexpr int col_threads(int n, int emax, int F) {
    return 2 * F * fft_TPF(n, emax) <= 512 ? (2 * F * fft_TPF(n, emax) < 32 ? 32 : 2 * F * fft_TPF(n, emax))
                                            : F * fft_TPF(n, emax);
}
inline int fft_smem_elems_h(int n, int F) { return (n + n / 16) * F; }

}  // namespace pss

/*
 * pss_oracle.h -- FP64 CPU oracle for the pseudo-spectral, semi-implicit
 * Euler-Maruyama step of a stochastic PDE on a periodic lattice (cuPSS,
 * arXiv:2405.02410, section "What cuPSS calculates").
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA path.
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * may load it.  It shares no code, header, table or constant with the CUDA
 * library, and the CUDA library never calls it.
 *
 * Conventions (the paper states them for the continuum only; the discrete
 * readings are listed in the design notes):
 *   - lattice sizes n[0] = Nx (contiguous axis), n[1] = Ny, n[2] = Nz; an unused
 *     axis has size 1.  Real arrays are [Nz][Ny][Nx], x fastest.
 *   - spectra are FULL complex arrays [Nz][Ny][Nx] (interleaved re, im) in
 *     standard FFT order: index k in 0..N-1 is the signed wavenumber k (k < N/2)
 *     or k - N (k >= N/2).
 *   - forward DFT is unnormalised, X_q = sum_x x e^{-i q.x}; the inverse
 *     carries 1/N_sites.
 */
#ifndef PSS_ORACLE_H
#define PSS_ORACLE_H
#include <stdint.h>

#define ORC_MAX_MONO 8

/* One dynamic field and its equation, "dt phi + O(q) phi = M(q) F[(F^-1[m phi])^p]"
 * plus noise of strength D~(q) = D (q^2)^noise_pow ("Writing models" and
 * "Adding noise" sections). */
typedef struct {
    int dim;                /* 1, 2 or 3 */
    int n[3];               /* Nx, Ny, Nz (unused axes = 1) */
    double dx[3];           /* lattice spacings (unused axes: 1) */
    double dt;              /* time step */
    uint64_t seed;          /* Philox key */
    int field_id;           /* Philox counter word 2 */
    int n_lhs;              /* implicit operator O(q) = sum lhs_coef[m] (q^2)^lhs_pow[m]; L(q) = -O(q) */
    double lhs_coef[ORC_MAX_MONO];
    int lhs_pow[ORC_MAX_MONO];
    int n_rhs;              /* explicit operator M(q) = sum rhs_coef[m] (q^2)^rhs_pow[m] */
    double rhs_coef[ORC_MAX_MONO];
    int rhs_pow[ORC_MAX_MONO];
    int power;              /* order p of the product phi^p (0: no explicit term) */
    int noisy;              /* 0: deterministic */
    double noise_D;         /* D in D~(q) = D (q^2)^noise_pow */
    int noise_pow;
    int dealias_order;      /* n_d: keep iff (n_d+1)|k_j| < N_j on every axis; 0 keeps all */
    int transform;          /* 0: auto (naive DFT for N_sites <= 256), 1: naive DFT, 2: radix-2 FFT */
    int grad2;              /* 1: the product is |grad(m phi)|^2 = sum_j (F^-1[i q_j m phi])^2 (the KPZ
                               nonlinearity with psi = grad phi) instead of (F^-1[m phi])^power; power = 2.
                               q_j of a Nyquist index is 0 (the derivative of a real field stays real) */
} orc_field;

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* u = ((x >> 8) + 0.5) / 2^24, strictly inside (0, 1). */
double orc_uniform24(uint32_t x);
/* Box-Muller pair from Philox(ctr = (c0, c1, c2, c3), key = seed): from
 * output words (x0, x1), or (x2, x3) when upper != 0. */
void orc_normal_pair(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                     double *n1, double *n2);
void orc_normal_pair_words(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                           int upper, double *n1, double *n2);

/* In-place d-dimensional complex transform of data[2*N_sites]; sign = -1
 * forward, +1 inverse (both unnormalised).  method: 1 naive DFT, 2 radix-2 FFT. */
int orc_dft(int dim, const int n[3], double *data, int sign, int method);

/* Dealias mask value (0 or 1) of full-spectrum mode (kx, ky, kz). */
int orc_mask(const orc_field *f, int kx, int ky, int kz);
/* q^2 of full-spectrum mode (kx, ky, kz). */
double orc_q2(const orc_field *f, int kx, int ky, int kz);

/* P_q = F[ (F^-1[m phi])^p ] for a full spectrum phi (Eq. nonlin_general without M),
 * or F[ sum_j (F^-1[i q_j m phi])^2 ] when grad2 is set. */
int orc_nonlinear(const orc_field *f, const double *phi, double *P);
/* Noise increment xi_q of time step `step` (full spectrum), i.e. sqrt(dt) eta~_q of Eq. timeupdate.
 * Counter (((kz Ny + ky) Hxe + kx) / 2, step, field_id, 0) of the canonical
 * member (kx, ky, kz) of the Hermitian pair, Hxe = Nx/2+1 rounded up to even;
 * words (x0, x1) for even kx, (x2, x3) for odd kx. */
int orc_noise(const orc_field *f, int64_t step, double *xi);
/* nsteps steps of Eq. timeupdate on the full spectrum phi, steps step0 .. step0+nsteps-1. */
int orc_run(const orc_field *f, double *phi, int64_t step0, int64_t nsteps);
/* Initial real field phi_x = lo + (hi - lo) u(Philox(seed, (site, 0, field_id, 1))). */
int orc_init_uniform(const orc_field *f, double lo, double hi, double *phi_real);
/* Radially binned structure factor S(q) = |phi_q|^2 / N_sites over (0, q_max],
 * q_max = pi / dx[0], nbins equal bins; S_out[nbins], count_out[nbins] (modes per bin),
 * *L_out = 2 pi sum S / sum |q| S over the binned modes. */
int orc_structure_factor(const orc_field *f, const double *phi, int nbins,
                         double *S_out, double *count_out, double *L_out);

/* Adjoint of orc_run(f, phi, step0, nsteps) at phi0 (full spectrum).  On entry
 * lambda holds dJ/dphi_T, on exit dJ/dphi_0, both for the inner product
 * <a, b> = Re sum conj(a) b over the full spectrum.  grad[0..4] receives
 * dJ/dO_k (the implicit coefficient of (q^2)^k), grad[5..9] dJ/dM_k, grad[10]
 * dJ/dD.  Power products only (grad2 = 0; else returns -3).  Keeps every intermediate state (nsteps + 1 spectra). */
int orc_adjoint(const orc_field *f, const double *phi0, int64_t step0, int64_t nsteps, double *lambda,
                double *grad);

#endif

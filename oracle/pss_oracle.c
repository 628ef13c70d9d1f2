/*
 * pss_oracle.c -- plain FP64 CPU oracle for one time step of the cuPSS method
 * (arXiv:2405.02410).
 *
 * TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
 * CPU-baseline leg are its only users.  It shares nothing with the CUDA
 * library and is deliberately slow and literal.
 *
 * What it follows:
 *   - Eq. (timeupdate), section "What cuPSS calculates": semi-implicit
 *     Euler-Maruyama update phi <- (phi + dt sum N + sqrt(dt) eta~) / (1 - dt L~).
 *   - The six numbered steps of that section, in that order: intermediate
 *     terms (none here: the factor is the field itself), de-alias, go to real
 *     space and multiply, go back to Fourier space, draw noise, update.
 *   - Eq. (nonlin_general) / Eq. (cubicexampledealiased): N = M(q) F[(F^-1[phi^d])^p].
 *   - Section "De-aliasing": a field in an order-n nonlinearity loses modes with
 *     |q| > 2 pi / ((n+1) dx); read per axis as (n+1)|k_j| < N_j.
 *   - Eq. (noise_eq) and "Adding noise": <eta eta> = 2 D~(q) (2pi)^d delta delta,
 *     D~ = D (q^2)^m (D q^2 is the conserved-current noise of the Introduction).
 *   - the fields are real (Eq. basereal): after each update only the Hermitian
 *     part of the spectrum is kept (see hermitian_part).
 *
 * Parity pins for every function are in tests/test_oracle_*.py.
 */
#include "pss_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from the published definition (Salmon et al., SC'11):     */
/* 10 rounds of two 32x32->64 multiplies; Weyl key schedule.                */
/* ------------------------------------------------------------------------ */
static uint32_t mulhi32(uint32_t a, uint32_t b)
{
    return (uint32_t)(((uint64_t)a * (uint64_t)b) >> 32);
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;   /* round multipliers */
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;   /* key increments */
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint32_t hi0 = mulhi32(M0, c0), lo0 = M0 * c0;
        uint32_t hi1 = mulhi32(M1, c2), lo1 = M1 * c2;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

double orc_uniform24(uint32_t x)
{
    return ((double)(x >> 8) + 0.5) / 16777216.0;
}

void orc_normal_pair(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                     double *n1, double *n2)
{
    orc_normal_pair_words(seed, c0, c1, c2, c3, 0, n1, n2);
}

void orc_normal_pair_words(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                           int upper, double *n1, double *n2)
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t x[4];
    orc_philox4x32_10(ctr, key, x);
    double u0 = orc_uniform24(x[upper ? 2 : 0]);
    double u1 = orc_uniform24(x[upper ? 3 : 1]);
    /* Box-Muller transform */
    double r = sqrt(-2.0 * log(u0));
    *n1 = r * cos(2.0 * M_PI * u1);
    *n2 = r * sin(2.0 * M_PI * u1);
}

/* ------------------------------------------------------------------------ */
/* Transforms (the F and F^-1 of Eq. cubicexample).                         */
/* ------------------------------------------------------------------------ */

/* Naive O(n^2) DFT of one line: X_k = sum_j x_j exp(sign 2 pi i j k / n). */
static void dft_naive_line(double *re, double *im, int n, int sign)
{
    double *xr = malloc(sizeof(double) * (size_t)n);
    double *xi = malloc(sizeof(double) * (size_t)n);
    for (int k = 0; k < n; ++k) {
        double sr = 0.0, si = 0.0;
        for (int j = 0; j < n; ++j) {
            long m = ((long)j * (long)k) % n;        /* exact angle reduction */
            double ang = sign * 2.0 * M_PI * (double)m / (double)n;
            double c = cos(ang), s = sin(ang);
            sr += re[j] * c - im[j] * s;
            si += re[j] * s + im[j] * c;
        }
        xr[k] = sr;
        xi[k] = si;
    }
    memcpy(re, xr, sizeof(double) * (size_t)n);
    memcpy(im, xi, sizeof(double) * (size_t)n);
    free(xr);
    free(xi);
}

/* Iterative radix-2 decimation-in-time FFT of one line (n a power of two):
 * bit-reversal permutation, then log2(n) stages of butterflies with twiddles
 * exp(sign 2 pi i m / len) evaluated directly from cos/sin. */
static void fft_radix2_line(double *re, double *im, int n, int sign)
{
    for (int i = 1, j = 0; i < n; ++i) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double t = re[i]; re[i] = re[j]; re[j] = t;
            t = im[i]; im[i] = im[j]; im[j] = t;
        }
    }
    for (int len = 2; len <= n; len <<= 1) {
        int half = len >> 1;
        for (int m = 0; m < half; ++m) {
            double ang = sign * 2.0 * M_PI * (double)m / (double)len;
            double wr = cos(ang), wi = sin(ang);
            for (int s = 0; s < n; s += len) {
                int a = s + m, b = s + m + half;
                double tr = re[b] * wr - im[b] * wi;
                double ti = re[b] * wi + im[b] * wr;
                re[b] = re[a] - tr; im[b] = im[a] - ti;
                re[a] = re[a] + tr; im[a] = im[a] + ti;
            }
        }
    }
}

static int is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

int orc_dft(int dim, const int n[3], double *data, int sign, int method)
{
    int N[3] = {n[0], dim > 1 ? n[1] : 1, dim > 2 ? n[2] : 1};
    long stride[3] = {1, N[0], (long)N[0] * N[1]};
    long nsites = (long)N[0] * N[1] * N[2];
    int maxn = N[0] > N[1] ? N[0] : N[1];
    if (N[2] > maxn) maxn = N[2];
    double *re = malloc(sizeof(double) * (size_t)maxn);
    double *im = malloc(sizeof(double) * (size_t)maxn);
    for (int ax = 0; ax < 3; ++ax) {
        int len = N[ax];
        if (len == 1) continue;
        if (method == 2 && !is_pow2(len)) { free(re); free(im); return -1; }
        for (long base = 0; base < nsites; ++base) {
            /* a line along axis ax starts at every site whose ax-coordinate is 0 */
            if ((base / stride[ax]) % len != 0) continue;
            for (int j = 0; j < len; ++j) {
                re[j] = data[2 * (base + j * stride[ax])];
                im[j] = data[2 * (base + j * stride[ax]) + 1];
            }
            if (method == 1) dft_naive_line(re, im, len, sign);
            else fft_radix2_line(re, im, len, sign);
            for (int j = 0; j < len; ++j) {
                data[2 * (base + j * stride[ax])] = re[j];
                data[2 * (base + j * stride[ax]) + 1] = im[j];
            }
        }
    }
    free(re);
    free(im);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Lattice helpers                                                          */
/* ------------------------------------------------------------------------ */
static void dims(const orc_field *f, int N[3])
{
    N[0] = f->n[0];
    N[1] = f->dim > 1 ? f->n[1] : 1;
    N[2] = f->dim > 2 ? f->n[2] : 1;
}

static long n_sites(const orc_field *f)
{
    int N[3];
    dims(f, N);
    return (long)N[0] * N[1] * N[2];
}

static int transform_method(const orc_field *f)
{
    if (f->transform == 1 || f->transform == 2) return f->transform;
    return n_sites(f) <= 256 ? 1 : 2;
}

/* signed wavenumber of unsigned index k on an axis of length n; the Nyquist
 * index n/2 maps to -n/2 (q^2 does not depend on the choice) */
static int signed_k(int k, int n)
{
    return k < (n + 1) / 2 ? k : k - n;
}

double orc_q2(const orc_field *f, int kx, int ky, int kz)
{
    int N[3], k[3] = {kx, ky, kz};
    dims(f, N);
    double q2 = 0.0;
    for (int j = 0; j < 3; ++j) {
        if (N[j] == 1) continue;
        double qj = 2.0 * M_PI * (double)signed_k(k[j], N[j]) / ((double)N[j] * f->dx[j]);
        q2 += qj * qj;
    }
    return q2;
}

int orc_mask(const orc_field *f, int kx, int ky, int kz)
{
    int N[3], k[3] = {kx, ky, kz};
    dims(f, N);
    for (int j = 0; j < 3; ++j) {
        int a = abs(signed_k(k[j], N[j]));
        if ((long)(f->dealias_order + 1) * a >= N[j] && N[j] > 1) return 0;
    }
    return 1;
}

static double poly_q2(int nm, const double *coef, const int *pw, double q2)
{
    double s = 0.0;
    for (int m = 0; m < nm; ++m) s += coef[m] * pow(q2, (double)pw[m]);
    return s;
}

/* ------------------------------------------------------------------------ */
/* Step pieces                                                              */
/* ------------------------------------------------------------------------ */
/* q_j of unsigned index k on axis j for an odd (first-derivative) operator:
 * the Nyquist index of an even axis has q_j = 0 */
static double q_axis(const orc_field *f, int j, int k, int n)
{
    if (n % 2 == 0 && k == n / 2) return 0.0;
    return 2.0 * M_PI * (double)signed_k(k, n) / ((double)n * f->dx[j]);
}

/* |grad(m phi)|^2 in real space, back to Fourier space (section "Writing
 * models", the KPZ example: the nonlinearity lambda psi^2 with psi = grad phi) */
static int nonlinear_grad2(const orc_field *f, const double *phi, double *P)
{
    int N[3];
    dims(f, N);
    long ns = n_sites(f);
    int method = transform_method(f);
    double *D = malloc(sizeof(double) * (size_t)(2 * ns));
    if (!D) return -2;
    for (long i = 0; i < 2 * ns; ++i) P[i] = 0.0;
    for (int j = 0; j < f->dim; ++j) {
        /* psi_j = F^-1[i q_j m phi] */
        for (int kz = 0; kz < N[2]; ++kz)
            for (int ky = 0; ky < N[1]; ++ky)
                for (int kx = 0; kx < N[0]; ++kx) {
                    long i = ((long)kz * N[1] + ky) * N[0] + kx;
                    int k[3] = {kx, ky, kz};
                    double q = orc_mask(f, kx, ky, kz) ? q_axis(f, j, k[j], N[j]) : 0.0;
                    D[2 * i] = -q * phi[2 * i + 1];
                    D[2 * i + 1] = q * phi[2 * i];
                }
        if (orc_dft(f->dim, f->n, D, +1, method)) { free(D); return -1; }
        for (long i = 0; i < ns; ++i) {
            double r = D[2 * i] / (double)ns;
            P[2 * i] += r * r;
        }
    }
    free(D);
    return orc_dft(f->dim, f->n, P, -1, method);
}

int orc_nonlinear(const orc_field *f, const double *phi, double *P)
{
    int N[3];
    dims(f, N);
    long ns = n_sites(f);
    int method = transform_method(f);
    if (f->grad2) return nonlinear_grad2(f, phi, P);
    /* step 2: de-alias, d = m phi */
    for (int kz = 0; kz < N[2]; ++kz)
        for (int ky = 0; ky < N[1]; ++ky)
            for (int kx = 0; kx < N[0]; ++kx) {
                long i = ((long)kz * N[1] + ky) * N[0] + kx;
                int m = orc_mask(f, kx, ky, kz);
                P[2 * i] = m ? phi[2 * i] : 0.0;
                P[2 * i + 1] = m ? phi[2 * i + 1] : 0.0;
            }
    /* step 3: to real space (inverse carries 1/N_sites), product r^p */
    if (orc_dft(f->dim, f->n, P, +1, method)) return -1;
    for (long i = 0; i < ns; ++i) {
        double r = P[2 * i] / (double)ns;   /* the field is real: keep Re */
        double u = 1.0;
        for (int p = 0; p < f->power; ++p) u *= r;
        P[2 * i] = u;
        P[2 * i + 1] = 0.0;
    }
    /* step 4: back to Fourier space */
    return orc_dft(f->dim, f->n, P, -1, method);
}

int orc_noise(const orc_field *f, int64_t step, double *xi)
{
    int N[3];
    dims(f, N);
    long ns = n_sites(f);
    int Hx = N[0] / 2 + 1;
    double dV = 1.0;
    for (int j = 0; j < f->dim; ++j) dV *= f->dx[j];
    for (int kz = 0; kz < N[2]; ++kz)
        for (int ky = 0; ky < N[1]; ++ky)
            for (int kx = 0; kx < N[0]; ++kx) {
                long i = ((long)kz * N[1] + ky) * N[0] + kx;
                xi[2 * i] = 0.0;
                xi[2 * i + 1] = 0.0;
                if (!f->noisy) continue;
                /* The real field makes xi_{-q} = conj(xi_q).  Each pair is drawn
                 * once, by its member with the smaller index in the half
                 * spectrum [kz][ky][0..Nx/2]; a mode equal to its own partner
                 * is real. */
                int pkx = (N[0] - kx) % N[0], pky = (N[1] - ky) % N[1], pkz = (N[2] - kz) % N[2];
                long own = kx <= N[0] / 2 ? ((long)kz * N[1] + ky) * Hx + kx : -1;
                long par = pkx <= N[0] / 2 ? ((long)pkz * N[1] + pky) * Hx + pkx : -1;
                long canon;
                int conj;
                int ckx, cky, ckz;   /* the canonical member */
                if (own < 0) { canon = par; conj = 1; }
                else if (par < 0) { canon = own; conj = 0; }
                else { canon = own < par ? own : par; conj = canon != own; }
                if (canon == own) { ckx = kx; cky = ky; ckz = kz; }
                else { ckx = pkx; cky = pky; ckz = pkz; }
                int selfconj = own >= 0 && own == par;
                /* One Philox call serves the canonical modes kx = 2j and 2j + 1
                 * of a row: counter word 0 = ((kz Ny + ky) Hxe + kx) / 2 with
                 * Hxe = Nx/2+1 rounded up to even; words (x0, x1) feed even kx,
                 * (x2, x3) odd kx. */
                long Hxe = Hx + (Hx & 1);
                long pairidx = (((long)ckz * N[1] + cky) * Hxe + ckx) >> 1;
                double q2 = orc_q2(f, kx, ky, kz);
                double Dq = f->noise_D * pow(q2, (double)f->noise_pow);
                if (f->noise_pow > 0 && q2 == 0.0) Dq = 0.0;
                /* per-component variance N_sites D~ dt / dV: the lattice form of
                 * 2 D~ (2pi)^d delta(q+q') delta(t-t') integrated over one step */
                double sigma = sqrt((double)ns * Dq * f->dt / dV);
                double n1, n2;
                orc_normal_pair_words(f->seed, (uint32_t)pairidx, (uint32_t)step, (uint32_t)f->field_id, 0u,
                                      ckx & 1, &n1, &n2);
                if (selfconj) {
                    xi[2 * i] = sqrt(2.0) * sigma * n1;
                    xi[2 * i + 1] = 0.0;
                } else {
                    xi[2 * i] = sigma * n1;
                    xi[2 * i + 1] = conj ? -sigma * n2 : sigma * n2;
                }
            }
    (void)ns;
    return 0;
}

/* The field is real (Eq. basereal), so its spectrum is Hermitian,
 * phi(-q) = conj phi(q).  Rounding in the transforms breaks that in the last
 * bit; the broken (anti-Hermitian) part is the spectrum of an imaginary field,
 * which the real-space product never sees, so a mode with |1 - dt L| < 1
 * would amplify it without bound.  After each update keep the Hermitian part. */
static void hermitian_part(const orc_field *f, double *phi)
{
    int N[3];
    dims(f, N);
    for (int kz = 0; kz < N[2]; ++kz)
        for (int ky = 0; ky < N[1]; ++ky)
            for (int kx = 0; kx < N[0]; ++kx) {
                long i = ((long)kz * N[1] + ky) * N[0] + kx;
                long j = ((long)((N[2] - kz) % N[2]) * N[1] + (N[1] - ky) % N[1]) * N[0] + (N[0] - kx) % N[0];
                if (j < i) continue;
                if (j == i) { phi[2 * i + 1] = 0.0; continue; }
                double re = 0.5 * (phi[2 * i] + phi[2 * j]);
                double im = 0.5 * (phi[2 * i + 1] - phi[2 * j + 1]);
                phi[2 * i] = re; phi[2 * i + 1] = im;
                phi[2 * j] = re; phi[2 * j + 1] = -im;
            }
}

int orc_run(const orc_field *f, double *phi, int64_t step0, int64_t nsteps)
{
    int N[3];
    dims(f, N);
    long ns = n_sites(f);
    double *P = calloc((size_t)(2 * ns), sizeof(double));
    double *xi = calloc((size_t)(2 * ns), sizeof(double));
    if (!P || !xi) { free(P); free(xi); return -2; }
    for (int64_t s = 0; s < nsteps; ++s) {
        int64_t step = step0 + s;
        /* steps 1-4: explicit term P_q = F[(F^-1[m phi])^p] */
        if (f->power > 0) {
            if (orc_nonlinear(f, phi, P)) { free(P); free(xi); return -1; }
        } else {
            memset(P, 0, sizeof(double) * (size_t)(2 * ns));
        }
        /* step 5: noise */
        orc_noise(f, step, xi);
        /* step 6: Eq. (timeupdate) with L = -O */
        for (int kz = 0; kz < N[2]; ++kz)
            for (int ky = 0; ky < N[1]; ++ky)
                for (int kx = 0; kx < N[0]; ++kx) {
                    long i = ((long)kz * N[1] + ky) * N[0] + kx;
                    double q2 = orc_q2(f, kx, ky, kz);
                    double O = poly_q2(f->n_lhs, f->lhs_coef, f->lhs_pow, q2);
                    double M = f->power > 0 ? poly_q2(f->n_rhs, f->rhs_coef, f->rhs_pow, q2) : 0.0;
                    double L = -O;
                    double den = 1.0 - f->dt * L;
                    phi[2 * i] = (phi[2 * i] + f->dt * M * P[2 * i] + xi[2 * i]) / den;
                    phi[2 * i + 1] = (phi[2 * i + 1] + f->dt * M * P[2 * i + 1] + xi[2 * i + 1]) / den;
                }
        hermitian_part(f, phi);
    }
    free(P);
    free(xi);
    return 0;
}

int orc_init_uniform(const orc_field *f, double lo, double hi, double *phi_real)
{
    long ns = n_sites(f);
    for (long s = 0; s < ns; ++s) {
        uint32_t ctr[4] = {(uint32_t)s, 0u, (uint32_t)f->field_id, 1u};
        uint32_t key[2] = {(uint32_t)(f->seed & 0xffffffffu), (uint32_t)(f->seed >> 32)};
        uint32_t x[4];
        orc_philox4x32_10(ctr, key, x);
        phi_real[s] = lo + (hi - lo) * orc_uniform24(x[0]);
    }
    return 0;
}

int orc_structure_factor(const orc_field *f, const double *phi, int nbins,
                         double *S_out, double *count_out, double *L_out)
{
    int N[3];
    dims(f, N);
    long ns = n_sites(f);
    double sumS = 0.0, sumQS = 0.0;
    for (int b = 0; b < nbins; ++b) { S_out[b] = 0.0; count_out[b] = 0.0; }
    for (int kz = 0; kz < N[2]; ++kz)
        for (int ky = 0; ky < N[1]; ++ky)
            for (int kx = 0; kx < N[0]; ++kx) {
                long i = ((long)kz * N[1] + ky) * N[0] + kx;
                int k[3] = {kx, ky, kz};
                /* s = |q| / (q_max / nbins), q_max = pi / dx[0]; each term is exact
                 * for power-of-two sizes and unit spacing */
                double s2 = 0.0;
                for (int j = 0; j < 3; ++j) {
                    if (N[j] == 1) continue;
                    double t = (2.0 * (double)nbins * (double)signed_k(k[j], N[j]) * f->dx[0]) /
                               ((double)N[j] * f->dx[j]);
                    s2 += t * t;
                }
                if (s2 == 0.0) continue;
                double s = sqrt(s2);
                if (s > (double)nbins) continue;
                int b = (int)ceil(s) - 1;
                double S = (phi[2 * i] * phi[2 * i] + phi[2 * i + 1] * phi[2 * i + 1]) / (double)ns;
                S_out[b] += S;
                count_out[b] += 1.0;
                sumS += S;
                sumQS += sqrt(orc_q2(f, kx, ky, kz)) * S;
            }
    for (int b = 0; b < nbins; ++b)
        if (count_out[b] > 0) S_out[b] /= count_out[b];
    *L_out = sumQS > 0 ? 2.0 * M_PI * sumS / sumQS : 0.0;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Adjoint of orc_run.                                                      */
/*                                                                          */
/* Gradients use the real inner product <a, b> = Re sum_q conj(a_q) b_q    */
/* over the full spectrum, so that dJ = <lambda, dphi>.  One forward step   */
/* phi' = H[g (phi + dt M P + xi)], g = 1/(1 + dt O), P = F[r^p],           */
/* r = Re F^-1[m phi], H the Hermitian part, has the adjoint                */
/*   mu      = g H[lambda']                                                 */
/*   nu      = dt M mu                                                      */
/*   s       = Re( N F^-1[nu] )          (F^dagger = N F^-1)                */
/*   w       = p r^(p-1) s                                                  */
/*   lambda  = mu + m F[w] / N           ((F^-1)^dagger = F / N)            */
/* and the coefficient gradients                                            */
/*   dJ/dO_k += -dt sum q^2k Re(conj(mu) phi')                              */
/*   dJ/dM_k +=  dt sum q^2k Re(conj(mu) P)                                 */
/*   dJ/dD   +=     sum      Re(conj(mu) xi) / (2 D)                        */
/* (O and M grouped by power k of q^2; xi is proportional to sqrt(D)).      */
/* ------------------------------------------------------------------------ */
int orc_adjoint(const orc_field *f, const double *phi0, int64_t step0, int64_t nsteps, double *lambda,
                double *grad)
{
    if (f->grad2) return -3;   /* the adjoint covers power products only */
    int N[3];
    dims(f, N);
    long ns = n_sites(f);
    int method = transform_method(f);
    size_t sz = (size_t)(2 * ns);
    double *states = malloc(sizeof(double) * sz * (size_t)(nsteps + 1));
    double *P = malloc(sizeof(double) * sz);
    double *r = malloc(sizeof(double) * sz);
    double *xi = malloc(sizeof(double) * sz);
    double *tmp = malloc(sizeof(double) * sz);
    if (!states || !P || !r || !xi || !tmp) {
        free(states); free(P); free(r); free(xi); free(tmp);
        return -2;
    }
    for (int k = 0; k < 11; ++k) grad[k] = 0.0;
    /* forward pass, every state kept */
    memcpy(states, phi0, sizeof(double) * sz);
    for (int64_t n = 0; n < nsteps; ++n) {
        memcpy(states + sz * (size_t)(n + 1), states + sz * (size_t)n, sizeof(double) * sz);
        if (orc_run(f, states + sz * (size_t)(n + 1), step0 + n, 1)) goto fail;
    }
    /* backward pass */
    for (int64_t n = nsteps - 1; n >= 0; --n) {
        const double *phi = states + sz * (size_t)n;
        const double *phin = states + sz * (size_t)(n + 1);
        hermitian_part(f, lambda);
        /* r = Re F^-1[m phi] and P = F[r^p] */
        for (int kz = 0; kz < N[2]; ++kz)
            for (int ky = 0; ky < N[1]; ++ky)
                for (int kx = 0; kx < N[0]; ++kx) {
                    long i = ((long)kz * N[1] + ky) * N[0] + kx;
                    int m = orc_mask(f, kx, ky, kz);
                    r[2 * i] = m ? phi[2 * i] : 0.0;
                    r[2 * i + 1] = m ? phi[2 * i + 1] : 0.0;
                }
        if (orc_dft(f->dim, f->n, r, +1, method)) goto fail;
        for (long i = 0; i < ns; ++i) {
            double x = r[2 * i] / (double)ns, u = 1.0;
            for (int p = 0; p < f->power; ++p) u *= x;
            r[2 * i] = x;
            r[2 * i + 1] = 0.0;
            P[2 * i] = u;
            P[2 * i + 1] = 0.0;
        }
        if (f->power > 0 && orc_dft(f->dim, f->n, P, -1, method)) goto fail;
        orc_noise(f, step0 + n, xi);
        /* mu, coefficient gradients, nu */
        for (int kz = 0; kz < N[2]; ++kz)
            for (int ky = 0; ky < N[1]; ++ky)
                for (int kx = 0; kx < N[0]; ++kx) {
                    long i = ((long)kz * N[1] + ky) * N[0] + kx;
                    double q2 = orc_q2(f, kx, ky, kz);
                    double O = poly_q2(f->n_lhs, f->lhs_coef, f->lhs_pow, q2);
                    double M = f->power > 0 ? poly_q2(f->n_rhs, f->rhs_coef, f->rhs_pow, q2) : 0.0;
                    double g = 1.0 / (1.0 + f->dt * O);
                    double mr = g * lambda[2 * i], mi = g * lambda[2 * i + 1];
                    double a_phi = mr * phin[2 * i] + mi * phin[2 * i + 1];     /* Re(conj(mu) phi') */
                    double a_P = f->power > 0 ? mr * P[2 * i] + mi * P[2 * i + 1] : 0.0;
                    double a_xi = mr * xi[2 * i] + mi * xi[2 * i + 1];
                    double q2k = 1.0;
                    for (int k = 0; k < 5; ++k) {
                        grad[k] += -f->dt * q2k * a_phi;
                        grad[5 + k] += f->dt * q2k * a_P;
                        q2k *= q2;
                    }
                    if (f->noisy && f->noise_D > 0.0) grad[10] += a_xi / (2.0 * f->noise_D);
                    lambda[2 * i] = mr;
                    lambda[2 * i + 1] = mi;
                    tmp[2 * i] = f->dt * M * mr;
                    tmp[2 * i + 1] = f->dt * M * mi;
                }
        if (f->power > 0) {
            /* s = Re(N F^-1[nu]) is the unnormalised inverse transform */
            if (orc_dft(f->dim, f->n, tmp, +1, method)) goto fail;
            for (long i = 0; i < ns; ++i) {
                double rp = 1.0;
                for (int p = 0; p < f->power - 1; ++p) rp *= r[2 * i];
                tmp[2 * i] = (double)f->power * rp * tmp[2 * i];
                tmp[2 * i + 1] = 0.0;
            }
            if (orc_dft(f->dim, f->n, tmp, -1, method)) goto fail;
            for (int kz = 0; kz < N[2]; ++kz)
                for (int ky = 0; ky < N[1]; ++ky)
                    for (int kx = 0; kx < N[0]; ++kx) {
                        long i = ((long)kz * N[1] + ky) * N[0] + kx;
                        if (!orc_mask(f, kx, ky, kz)) continue;
                        lambda[2 * i] += tmp[2 * i] / (double)ns;
                        lambda[2 * i + 1] += tmp[2 * i + 1] / (double)ns;
                    }
        }
    }
    free(states); free(P); free(r); free(xi); free(tmp);
    return 0;
fail:
    free(states); free(P); free(r); free(xi); free(tmp);
    return -1;
}

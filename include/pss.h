/*
 * pss.h -- C ABI of libpss, the GB300 (sm_103a) implementation of one time
 * step of the cuPSS pseudo-spectral method (arXiv:2405.02410) for stochastic
 * PDEs on periodic 1D/2D/3D lattices.
 *
 * The calls follow the paper's recipe for building a model (section "Writing
 * models"): create a system (lattice size, spacing, time step), add named
 * parameters, add fields, add the implicit ("lhs") and explicit ("rhs") terms
 * of each field's equation "dt phi + lhs = rhs", add noise, set an initial
 * condition, then evolve.  Equations are given as structured terms instead of
 * strings.
 *
 * One time step (section "What cuPSS calculates", Eq. timeupdate) of every
 * dynamic field phi:
 *     phi_q <- (phi_q + dt M(q) P_q + xi_q) / (1 + dt O(q))
 * with O(q) = sum_m c_m (q^2)^p_m the implicit operator (L~ = -O),
 * M(q) the explicit operator, P_q = F[(F^-1[m phi])^p] the pseudo-spectral
 * product of the de-aliased field (section "De-aliasing"), and xi_q the noise
 * of strength D~(q) = D (q^2)^r (Eq. noise_eq, section "Adding noise").
 *
 * Conventions
 *   - sizes: nx is the contiguous axis; every used axis is a power of two in
 *     [4, 1024]; unused axes are 1.  Real fields are [nz][ny][nx] row-major.
 *   - spectra exchanged with the caller are the R2C half spectrum
 *     [nz][ny][nx/2+1] of complex values (interleaved re, im), forward DFT
 *     unnormalised, inverse with 1/(nx ny nz).
 *   - precision PSS_F32: real fields float, spectra float2; PSS_F64: double,
 *     double2.  Arithmetic runs in that precision on the GPU.
 *   - "where" PSS_HOST: the pointer is host memory (copied synchronously);
 *     PSS_DEVICE: device memory of the system's device, used on the system's
 *     stream.
 *   - ownership: the system owns every device buffer it allocates; caller
 *     buffers are only read or written during the call.
 *   - errors: every call returns PSS_OK (0) or a negative pss_status and sets
 *     a message readable with pss_last_error().  Nothing throws across the
 *     ABI.  Errors found on the device (non-finite values) are reported by the
 *     next call that synchronises (pss_get_*, pss_sync).
 *   - thread safety: one handle must not be used from two threads at once.
 */
#ifndef PSS_H
#define PSS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pss_system pss_system;

typedef enum {
    PSS_OK = 0,
    PSS_EINVAL = -1,        /* bad argument */
    PSS_ENOMEM = -2,        /* device allocation failed */
    PSS_ECUDA = -3,         /* a CUDA call failed */
    PSS_ETIMEOUT = -4,      /* a bounded device wait ran out */
    PSS_ENONFINITE = -5,    /* a field became NaN or Inf */
    PSS_EUNSUPPORTED = -6   /* valid, but outside what this build implements */
} pss_status;

enum { PSS_F32 = 0, PSS_F64 = 1 };
enum { PSS_HOST = 0, PSS_DEVICE = 1 };

/* Create a system on the current CUDA device ("evolver(dim, Nx, Ny, dx, dy,
 * dt, output)" of section "Example").  dim in {1,2,3}; seed keys the Philox
 * generator of the noise and of pss_init_uniform; precision PSS_F32/PSS_F64.
 * *out receives the handle (NULL on failure). */
int pss_create_system(pss_system **out, int dim, int nx, int ny, int nz,
                      double dx, double dy, double dz, double dt,
                      uint64_t seed, int precision);
/* A batch of `batch` independent instances of one system (an ensemble of
 * noise realisations or a parameter sweep): same lattice, fields and terms,
 * instance b keyed by seeds[b] and with its own parameter values
 * (pss_set_param_batch).  Every step advances all instances; the per-field
 * calls (set/get/init/structure factor) act on the instance chosen with
 * pss_select_instance (default 0).  pss_create_system is a batch of one. */
int pss_create_batch(pss_system **out, int batch, int dim, int nx, int ny, int nz,
                     double dx, double dy, double dz, double dt,
                     const uint64_t *seeds, int precision);
int pss_batch_size(const pss_system *s);
int pss_select_instance(pss_system *s, int instance);

/* Free every device buffer and the handle.  NULL is accepted. */
int pss_destroy_system(pss_system *s);
/* Launch all further work on this cudaStream_t (NULL = legacy default
 * stream).  Work issued after the call is ordered after all work the system
 * issued before it, on whichever stream. */
int pss_set_stream(pss_system *s, void *cuda_stream);

/* Named scalar parameter ("addParameter", section "Writing models"); *id
 * receives its index; every instance starts with `value`.  A parameter may
 * be changed later with pss_set_param / pss_set_param_batch; the change
 * applies from the next step on.  pss_get_param reads the selected instance. */
int pss_add_param(pss_system *s, const char *name, double value, int *id);
int pss_set_param(pss_system *s, int id, double value);              /* all instances */
int pss_set_param_batch(pss_system *s, int id, const double *values); /* values[batch] */
int pss_get_param(pss_system *s, int id, double *value);

/* Add a field ("createField(name, dynamic)").  Only dynamic fields are
 * implemented (dynamic = 1; 0 returns PSS_EUNSUPPORTED).  At most 4 fields.
 * Fields start at zero.  Add fields before setting data: adding a field
 * reallocates the arrays (existing fields keep their values). */
int pss_add_field(pss_system *s, const char *name, int dynamic, int *field_id);

/* Add a term to the equation of field_id.  The term's operator is
 *     sum_{m < n_mono} scales[m] * param[param_ids[m]] * (q^2)^q2_pows[m]
 * (param_ids[m] < 0 means the factor 1), applied to prod_k field_k^powers[k].
 * implicit = 1: an lhs term of "dt phi + lhs = rhs"; it must be linear in the
 *   field itself (n_factors = 1, factor_fields[0] = field_id, powers[0] = 1).
 * implicit = 0: an rhs term, treated explicitly.  This build implements rhs
 *   terms whose product is a power 1..3 of the field itself; several rhs terms
 *   of one field must share that power (their operators add up).
 * q2_pows in [0, 4], n_mono <= 8. */
int pss_add_term(pss_system *s, int field_id, int implicit,
                 int n_mono, const int *param_ids, const double *scales, const int *q2_pows,
                 int n_factors, const int *factor_fields, const int *powers);

/* Add a product term  M(q) F[ prod_k psi_k^powers[k] ]  to the rhs of the
 * equation of field_id (Eq. basefourier; section "Writing models": a
 * nonlinearity M prod_k psi_k^n_k whose factors psi_k are fields acted on by
 * differential operators).  M(q) is built from the monomials as in
 * pss_add_term.  Factor k is psi_k = F^-1[op_k(q) m phi_{factor_fields[k]}]
 * with the de-alias mask m of that field and
 *     op_k(q) = (i q_{derivs[k]} if derivs[k] >= 0) * (-q^2)^laps[k],
 * derivs[k] in -1 (none), 0..dim-1 (x, y, z; q = 0 at a Nyquist index),
 * laps[k] in 0..2, powers[k] in 1..4, 1..8 factors; derivs or laps NULL
 * means all -1 or all 0.  Factors may name any field of the system (of the
 * same instance).  A field with product terms evaluates all its explicit
 * terms (its power product from pss_add_term too) through real space: per
 * factor its transform back, then the products, the sums of the terms that
 * share one operator, and the transforms forward.  Such systems run the
 * generic kernels; the adjoint returns PSS_EUNSUPPORTED for them. */
int pss_add_product_term(pss_system *s, int field_id, int n_mono, const int *param_ids, const double *scales,
                         const int *q2_pows, int n_factors, const int *factor_fields, const int *powers,
                         const int *derivs, const int *laps);

/* Add the rhs term  M(q) F[ |grad(m phi)|^2 ]  to the equation of field_id,
 * M(q) = sum_{m < n_mono} scales[m] * param[param_ids[m]] * (q^2)^q2_pows[m]
 * as in pss_add_term.  This is the KPZ nonlinearity lambda (grad phi)^2 of
 * section "Writing models", written there as lambda psi^2 with psi = grad phi:
 * each derivative i q_j m phi (q_j = 0 at a Nyquist index) goes to real
 * space, their squares add up, and the sum goes back to Fourier space: the
 * product terms M (d_j phi)^2 of every axis j (pss_add_product_term). */
int pss_add_grad_sq_term(pss_system *s, int field_id, int n_mono, const int *param_ids, const double *scales,
                         const int *q2_pows);

/* Noise of strength D~(q) = param[D_param_id] * (q^2)^q2_pow on field_id
 * ("addNoise(phi, D*q^2)", section "Adding noise").  q2_pow in [0, 4]. */
int pss_set_noise(pss_system *s, int field_id, int D_param_id, int q2_pow);

/* De-aliasing order n of field_id (section "De-aliasing"): the field enters
 * products with its modes kept iff (n+1)|k_j| < N_j on every axis.  Default 2
 * (the two-thirds rule); 0 keeps every mode. */
int pss_set_dealias(pss_system *s, int field_id, int order);

/* Boundary frame of field_id along x (section "Callback functions": a
 * callback that sets the real field near the boundary at the end of every
 * step).  At the end of every step the sites with x < width take lo_value
 * and the sites with x >= Nx - width take hi_value (every y and z, every
 * instance), and the field's spectrum is taken again from that real field.
 * width = 0 removes the frame; 0 <= width <= Nx/2, values finite, else
 * PSS_EINVAL.  While a field has a frame, every step of the system ends with
 * each field taken to real space and back (four transforms per step instead
 * of two), and the adjoint returns PSS_EUNSUPPORTED. */
int pss_set_frame(pss_system *s, int field_id, int width, double lo_value, double hi_value);

/* Copy a real field [nz][ny][nx] in (and transform it). */
int pss_set_field(pss_system *s, int field_id, const void *real, int where);
/* Set a real field to lo + (hi - lo) u, u = ((x >> 8) + 0.5) / 2^24 with x the
 * first word of Philox4x32-10(counter = (site, 0, field_id, 1), key = seed). */
int pss_init_uniform(pss_system *s, int field_id, double lo, double hi);

/* Advance every dynamic field by n >= 0 steps.  Asynchronous on the system's
 * stream.  Step k of the run draws noise with Philox counter word 1 = k. */
int pss_step(pss_system *s, int64_t n);
/* Advance n systems (for instance the size classes of an ensemble) by
 * `steps` steps each, replayed from one captured CUDA graph on systems[0]'s
 * stream (the other systems are moved to that stream).  Distinct systems
 * are independent branches of the graph, which the GPU may run side by
 * side; a system listed more than once takes its steps in list order.
 * Errors are reported on systems[0]. */
int pss_step_many(pss_system **systems, int n, int64_t steps);
/* Gradients by the hand-written adjoint of the step (single field, batch 1).
 * Inner product: dJ = Re sum_q conj(lambda_q) dphi_q over the full spectrum,
 * both lambda and phi given as half spectra (the other half follows from
 * Hermitian symmetry).  The noise realisation is the one of the forward run.
 * pss_adjoint_forward: advance n >= 1 steps from the current state, keeping
 *   a checkpoint every ceil(sqrt(n)) steps on the device.
 * pss_adjoint_backward: lambda_T = dJ/dphi_T (half spectrum) of a loss of the
 *   state after that run; returns dJ/dparams[i] for every named parameter
 *   (operator coefficients and the noise strength; parameters not used by
 *   the field read 0) and, if lambda_0 != NULL, dJ/dphi_0 (half spectrum).
 *   Recomputes each segment forward from its checkpoint; accumulates the
 *   parameter gradients in FP64.  Leaves the state and step counter as after
 *   the forward run.  Synchronises. */
int pss_adjoint_forward(pss_system *s, int64_t n);
int pss_adjoint_backward(pss_system *s, const void *lambda_T, int where, double *dJ_dparams,
                         void *lambda_0, int where0);

/* Measurement: take n >= 1 steps like pss_step, but launch every kernel on
 * its own with a CUDA event pair around it, and return in avg_ms[0..3] the
 * mean duration (milliseconds) of each kind of launch of a step:
 * 0 = fused column kernel (update), 1 = inverse y pass (3D only),
 * 2 = row kernel (x transforms and product), 3 = forward y pass (3D only);
 * kinds that do not run read 0.  Synchronises. */
int pss_time_kernels(pss_system *s, int64_t n, double *avg_ms);

/* Launch-shape tuning (results do not depend on it).  key / value:
 *   "pdl"         1 = launch the step kernels with programmatic dependent
 *                 launch, 0 = plain stream order; by default on for the
 *                 kernels of the FP32 2D step below ("fast2d"), off for the
 *                 rest;
 *   "row_pairs"   row pairs per CTA of the x-transform kernel (power of two);
 *   "col_tiles"   column tiles per CTA of the fused column kernel;
 *   "mid_planes"  z planes per CTA of the 3D y-transform kernel;
 *   "graph_steps" steps per replayed CUDA graph;
 *   "col_radix", "row_radix", "mid_radix"
 *                 largest FFT pass radix (8 or 16) of the column, x and
 *                 3D y kernels;
 *   "fast2d"      FP32 2D systems whose sides are 256, 512 or 1024 points
 *                 run every transform in one warp (1, default) or take the
 *                 generic kernels (0); the two agree to FP32 rounding;
 *   "col2_warps"  warps beside the FFT groups of a column CTA of that path
 *                 that join its update (1..24);
 *   "row2_pairs"  row pairs per row CTA of that path (power of two <= 8);
 *   "adj_row_pairs" row pairs per CTA of the adjoint's x pass on that path
 *                 (power of two <= 8; automatic: the largest that still
 *                 gives every SM a CTA); the adjoint is the same bits;
 *   "row2_noise"  warps per row CTA of that path that draw the next step's
 *                 noise (1..24);
 *   "row2_share"  percentage (0..100) of that noise drawn by extra CTAs on
 *                 the SMs the row CTAs leave idle (default 0: none);
 *   "fast3d"      FP32 3D systems whose x side is 256, 512 or 1024 points
 *                 run their x pass on FFT groups (1, default) or on the
 *                 generic row kernel (0);
 *   "col2_radix", "row2_radix"
 *                 radix of that path's FFT passes (8 or 16);
 *   "real_state"  every step ends with each field taken to real space and
 *                 back, as with a boundary frame of width 0 (1; an ablation
 *                 of keeping the state in Fourier space, 0, default); the
 *                 two agree to rounding;
 *   "fuse_adjoint" the backward pass runs the last column part of one
 *                 adjoint step and the first of the step before it in one
 *                 launch (1, default, where its shared memory fits) or in
 *                 two (0); the adjoint fields agree bit for bit, the
 *                 gradients to the order of their FP64 atomic sums;
 *   "persist"     FP32 2D square systems of side 256, 512 or 1024 with
 *                 Model A/B or KPZ terms take a run of steps as one
 *                 cooperative launch with grid barriers between the column
 *                 and row phases (1, default) or as two launches a step on
 *                 the "fast2d" kernels (0); the same bits at the same FFT
 *                 radix;
 *   "persist_blocks" CTAs of that launch (0: automatic, one per SM and at
 *                 most one per column pair or row pair; values below the
 *                 smallest count that keeps every column and row pair in
 *                 shared memory are raised to it; at most the SMs);
 *   "persist_adj" on the persistent path, the backward pass of each
 *                 recomputed segment of pss_adjoint_backward runs as one
 *                 cooperative launch (1, default; the segment's forward run
 *                 then also keeps each step's noise) or as launches per
 *                 step (0); they agree to FP32 rounding;
 *   "adj_radix"   FFT pass radix of that persistent backward pass (8 or
 *                 16; 0, default: the forward step's);
 *   "adj_col2"    the column parts of the FP32 2D adjoint run on FFT groups,
 *                 one column pair per CTA (1, default) or on the generic
 *                 column kernel (0); they agree to FP32 rounding;
 *   "test_timeout" a check of the bounded device waits, for tests: with 1,
 *                 the first CTA of the generic column kernel expects 16
 *                 bytes more than its bulk copies deliver, and the first
 *                 CTA of the persistent step never arrives at its first
 *                 grid barrier; every wait gives up after 1024 polls (a few
 *                 milliseconds), so the next synchronising call returns
 *                 PSS_ETIMEOUT and clears the barrier words; results of the
 *                 steps taken meanwhile are wrong; 0 (default) turns it off;
 * 0 restores the automatic choice.  Unknown keys return PSS_EINVAL. */
int pss_set_tuning(pss_system *s, const char *key, int value);

/* Launch-shape autotuner: chooses the FFT pass radices, CTA tilings, noise
 * warps, programmatic dependent launch and steps per graph of this system's
 * step path by timing them on the GPU (the paper leaves launch shapes to the
 * library; they do not change results beyond the rounding order of the FFT
 * radix).  Coordinate descent: every knob of the path in turn takes each
 * value of its list with the others at their best so far, and a value is
 * kept only if its run is more than 1 % faster; each trial times at least
 * steps_per_trial steps (a whole number of graph replays) three times and
 * keeps the fastest.  Finally the starting settings and the result are
 * timed back to back, twice each; the result is kept only if it is not
 * slower there.
 *
 * The trials advance the system: its spectral state and step counter are
 * saved first (one temporary device copy of the state, allocated and freed
 * here) and restored afterwards, so the run continues as if the call had not
 * been made (the next step's product and noise are recomputed from the
 * restored state).  Cost: about 4 + (sum of the list lengths) trials of
 * (3 steps_per_trial + one graph) steps; synchronises.
 *
 * The chosen settings stay in force as pss_set_tuning values.  If report is
 * not NULL, a text of at most report_len bytes (NUL-terminated) describes
 * the outcome: "path=P trials=T skipped=S initial_ms=X tuned_ms=Y
 * key=value ...", with T the timed trials, S the values skipped because the
 * launcher refused them for this system (shared memory that would not fit),
 * X and Y the milliseconds per step of the starting and the chosen settings
 * and every knob of the path as its pss_set_tuning value (0 = automatic;
 * for "pdl", -1 = automatic).  Errors: PSS_EINVAL (NULL handle, no fields,
 * steps_per_trial < 1), a failing trial's status (state still restored). */
int pss_autotune(pss_system *s, int64_t steps_per_trial, char *report, size_t report_len);

/* Steps taken so far (the next step's noise index). */
int pss_get_step(pss_system *s, int64_t *step);
int pss_set_step(pss_system *s, int64_t step);

/* Real field [nz][ny][nx] out (synchronises; reports device-side errors). */
int pss_get_field(pss_system *s, int field_id, void *real_out, int where);
/* Half spectrum [nz][ny][nx/2+1] out / in. */
int pss_get_spectrum(pss_system *s, int field_id, void *half_out, int where);
int pss_set_spectrum(pss_system *s, int field_id, const void *half_in, int where);

/* Checkpoint and resume (the paper's runs write their state out at output
 * steps, section "Example"; this is the whole state a step reads).
 * pss_save_state writes into the host buffer buf: a header (format tag,
 * lattice, precision, batch, number of fields and parameters, step counter),
 * the parameter values of every instance [batch][nparams] (double), the
 * per-instance seeds [batch] (uint64) and the half spectrum of every field of
 * every instance [batch][nfields][nz][ny][nx/2+1] (the system's precision).
 * With buf == NULL only *len is set to the size needed; with *len smaller
 * than that, PSS_EINVAL and *len set to the size.  On success *len is the
 * size written.  Synchronises.
 * pss_load_state restores such a buffer into a system built the same way
 * (same lattice, precision, batch, number of fields and parameters; else
 * PSS_EINVAL and nothing changes): spectra, step counter, parameter values
 * and seeds.  The next step's nonlinear product and noise are recomputed
 * from the loaded state, so a resumed run takes the same steps, bit for bit,
 * as one that was never interrupted.  Launch-shape settings (pss_set_tuning)
 * are not part of the state.  Synchronises. */
int pss_save_state(pss_system *s, void *buf, size_t *len);
int pss_load_state(pss_system *s, const void *buf, size_t len);

/* Radially binned structure factor S(q) = |phi_q|^2 / N_sites over
 * 0 < |q| <= pi/dx, nbins equal bins (b = ceil(|q| nbins dx / pi) - 1), over
 * the full Hermitian set of modes; S_out[nbins] are bin means (FP64 sums),
 * count_out[nbins] (may be NULL) the modes per bin, *L_out (may be NULL) the
 * length 2 pi sum S / sum |q| S.  Host pointers; synchronises. */
int pss_structure_factor(pss_system *s, int field_id, int nbins,
                         double *S_out, double *count_out, double *L_out);

/* The same binned structure factor as pss_structure_factor, computed without
 * allocating any memory.  The paper has no counterpart: this is a library
 * service for callers that must not allocate while they run, such as a
 * process whose device memory is handed out up front by another allocator
 * (a late cudaMalloc there fails or fragments the pool), or a loop that
 * cannot afford cudaFree, which waits for the whole device and so stalls
 * work on every stream.  pss_structure_factor may grow its accumulator
 * with cudaFree + cudaMalloc; this entry point never does.
 *
 * The FP64 bin accumulator is a fixed array of 2 * PSS_NOALLOC_MAX_BINS + 2
 * doubles (16.4 KB) inside the library, present on every GPU that loads the
 * library until the process exits.  nbins must lie in
 * [1, PSS_NOALLOC_MAX_BINS]; larger requests fail with PSS_EINVAL and touch
 * nothing.  The system's device must be the current device.
 *
 * The first call on a device looks up the array's device address (set-up,
 * once per device); make that first call before any stream capture.
 *
 * Every call, from every system on the device, shares the one array; each
 * call clears the part it uses before accumulating and synchronises the
 * system's stream before returning.  Calls whose GPU work overlaps (two
 * host threads calling on different streams at once) race on the array and
 * return wrong sums: serialise them.
 *
 * Arguments, outputs and errors are those of pss_structure_factor. */
#define PSS_NOALLOC_MAX_BINS 1024
int pss_structure_factor_noalloc(pss_system *s, int field_id, int nbins,
                                 double *S_out, double *count_out, double *L_out);

/* Wait for the system's stream and report device-side errors. */
int pss_sync(pss_system *s);

/* Message of the last failed call on this handle (valid until the next
 * call).  pss_last_error(NULL) returns the message of a failed create. */
const char *pss_last_error(const pss_system *s);

/* Number of kernel launches this handle has issued (a count kept by the
 * host; for measurement). */
int64_t pss_launch_count(const pss_system *s);

/* Which kernels a step of this system runs (for measurement and profiling):
 * 1 = the FP32 2D kernels with one FFT group per transform (k2_col, k2_row:
 * FP32 2D systems with sides of 256, 512 or 1024 points, unless the tuning
 * key "fast2d" is 0); 2 = the generic 3D kernels with the x pass on FFT
 * groups (k_col, k_mid, k2_row: FP32 3D systems whose x side is 256, 512 or
 * 1024 points, unless "fast3d" is 0); 0 = the generic kernels (k_col,
 * k_mid, k_row).  Returns PSS_EINVAL for a NULL handle. */
int pss_step_path(const pss_system *s);

#ifdef __cplusplus
}
#endif
#endif

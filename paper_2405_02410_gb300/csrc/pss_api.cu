// pss_api.cu -- host side of libpss: the C ABI declared in include/pss.h.
//
// A system holds `batch` independent instances of one lattice problem.  Each
// (instance, field) pair is a slot; the spectral state phi_q of all slots and
// two work arrays A, B live back to back in three device buffers (tiled
// layout, see pss_internal.h).  B carries the x-transformed nonlinear
// product from one step to the next; A holds the inverse-transformed
// de-aliased field inside a step.  Per-slot parameters (operators, noise
// amplitude, mask, seed) live in a device array that is refreshed before
// launches, so runs of steps replay one captured CUDA graph even when
// parameters change between runs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/pss.h"
#include "pss_internal.h"

using namespace pss;

namespace {

struct Mono {
    int param;       // < 0: factor 1
    double scale;
    int pow;
};

struct Field {
    std::string name;
    std::vector<Mono> lhs, rhs;
    int power = 0;
    bool noisy = false;
    int noise_param = -1;
    int noise_pow = 0;
    int dealias = 2;
    bool general = false;              // has product terms (evaluated through real space)
    int frame_w = 0;                   // boundary frame along x (0: none)
    double frame_lo = 0, frame_hi = 0;
};

// One factor psi^power of a product term: psi = F^-1[op(q) m phi_field],
// op(q) = (i q_deriv if deriv >= 0) (-q^2)^lap.
struct GFactor {
    int field, power, deriv, lap;
};
// M(q) F[prod_k psi_k^n_k] on the rhs of field `target`.
struct GTerm {
    int target;
    std::vector<Mono> M;
    std::vector<GFactor> factors;
};

constexpr int kDefaultGraphSteps = 16;
constexpr int kTestWaitLimit = 1024;   // polls of a wait under the "test_timeout" check (a few ms)
constexpr int kMaxBatch = 65535 / kMaxFields;
constexpr double kPi = 3.14159265358979323846;

}  // namespace

struct pss_system {
    int dim = 0, nx = 1, ny = 1, nz = 1;
    double dx[3] = {1, 1, 1};
    double dt = 0;
    int batch = 1;
    std::vector<uint64_t> seeds;             // per instance
    int prec = PSS_F32;
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    std::vector<std::string> param_names;
    std::vector<double> param_values;        // [instance][param]
    std::vector<Field> fields;
    std::vector<GTerm> gterms;               // product terms (pss_add_product_term, pss_add_grad_sq_term)
    int cur = 0;                             // instance addressed by the per-field calls
    int hx = 0, ntiles = 0, rows = 0, n_outer = 1, n_inner = 1;
    long long nsites = 0;
    size_t field_elems = 0;                  // complex elements of one slot of one array
    void *state = nullptr, *A = nullptr, *B = nullptr;   // [slot][field_elems]
    void *XI = nullptr;                      // fast 2D path: unit-amplitude noise of the next step [slot][field_elems]
    void *fps = nullptr;                     // FieldP<T>[slots] on the device
    bool fps_dirty = true;
    void *tw = nullptr;                      // roots of unity, precision of the system
    void *real = nullptr;                    // real scratch [nz][ny][nx] (one slot)
    void *GS = nullptr;                      // product terms: factor / product spectrum [slot][field_elems]
    void *real_acc = nullptr;                // product terms: sum of the products in real space (one slot)
    void *real_tp = nullptr;                 // product terms: running product of one term (one slot)
    void *half = nullptr;                    // half-spectrum scratch (one slot)
    double *sq = nullptr;                    // structure-factor accumulator
    int sq_cap = 0;
    long long *d_step = nullptr;
    int *d_status = nullptr;
    int64_t step = 0;
    bool stale = true;                       // B does not hold the product of the current state
    bool b_fast = false;                     // B is in the column-major layout of the fast 2D path
    // captured step graphs by length (graphs[n]: n steps); all of them are
    // dropped when the launches they hold change (invalidate)
    std::vector<cudaGraphExec_t> graphs;
    bool graph_valid = false;
    uint64_t gen = 0;                        // bumped by every invalidation (pss_step_many's cache)
    uint64_t uid = 0;                        // unique per handle of the process (never reused)
    // pss_step_many's graphs with this system first: the systems (by uid and
    // generation at capture) and the number of steps of each
    struct Many {
        std::vector<uint64_t> uids, gens;
        int len = 0;
        cudaGraphExec_t exec = nullptr;
        int64_t stamp = 0;
    };
    std::vector<Many> many;
    int64_t many_clock = 0;
    // launch-shape tuning (pss_set_tuning); 0 = automatic
    int tune_pdl = -1, tune_row_pairs = 0, tune_col_tiles = 0, tune_graph_steps = 0, tune_mid_planes = 0;
    int tune_col_radix = 0, tune_row_radix = 0, tune_mid_radix = 0;   // FFT radix caps (8 or 16; 0 = automatic)
    int tune_fast2d = 1;                     // FP32 2D sides of 256..1024: one warp per transform (0 = generic kernels)
    int tune_col2_warps = 0, tune_row2_pairs = 0;   // its noise warps per column CTA, row pairs per row CTA
    int tune_col2_radix = 0, tune_row2_radix = 0;   // its FFT pass radix (8 or 16; 0 = automatic)
    int tune_row2_noise = 0;                 // noise warps per row CTA of that path (0 = automatic)
    int tune_adj_row_pairs = 0;              // row pairs per CTA of the adjoint's FFT-group x pass (0 = automatic)
    int tune_real_state = 0;                 // every step ends in real space and comes back (ablation)
    int tune_fuse_adj = 1;                   // adjoint: one launch for part B of a step and part A of the one before
    int tune_row2_share = -1;                // % of the noise drawn by extra CTAs on idle SMs (-1 = automatic: 0)
    int num_sms = 0;
    int tune_fast3d = 1;                     // FP32 3D x pass with one FFT group per row pair (0 = generic k_row)
    int tune_test_timeout = 0;               // check of the bounded waits: one CTA's wait runs out (tests)
    int tune_persist = 1;                    // square FP32 2D systems: a run of steps as one persistent launch
    int tune_adj_col2 = 1;
    int tune_adj_radix = 0;                  // FFT radix of that backward pass (8 or 16; 0: the forward's)
    int tune_persist_adj = 1;                // FP32 2D adjoint on the persistent path: a segment's backward pass in one launch                   // FP32 2D adjoint: column parts on FFT groups (0: generic kernel)
    int tune_persist_blocks = 0;             // its CTAs (0: every SM, at most one CTA per column pair or row pair)
    int coop = 0;                            // the device takes cooperative launches
    // captured persistent launches by run length (one kernel node each); p2_capture < 0: capture
    // of the cooperative launch is refused here, launch directly
    std::vector<std::pair<int, cudaGraphExec_t>> p2_graphs;
    int p2_capture = 1;
    GridSync *gs = nullptr;                  // grid-barrier words of the persistent step
    int64_t launches = 0;
    std::string err;
    // adjoint: checkpoints of the last pss_adjoint_forward run
    void *L = nullptr;                       // adjoint state lambda / mu (tiled, one slot)
    void *ck = nullptr;                      // checkpoints [nck + 1][slot]
    void *seg = nullptr;                     // recomputed states of one segment [K + 1][slot]
    void *seg_prod = nullptr;                // their x(y)-transformed products [K + 1][slot]
    void *seg_real = nullptr;                // their de-aliased real fields [K + 1][nsites]
    void *seg_noise = nullptr;               // their unit noise [K + 1][slot] (the persistent path)
    double *d_grad = nullptr;                // [11]
    long long *d_seg = nullptr;              // [2]: segment index, step of its first step (device)
    int64_t adj_n = 0, adj_step0 = 0, adj_K = 0, adj_nck = 0;
    bool adj_ready = false;
    cudaGraphExec_t adj_graph = nullptr;     // one full segment of the backward pass
    bool adj_graph_valid = false;
    int64_t adj_graph_launches = 0;

    int nslots() const { return batch * (int)fields.size(); }
    int64_t graph_launches = 0;              // launches per step of the captured step graph
};

namespace {

std::string g_create_err;

int fail(pss_system *s, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (s) s->err = buf;
    else g_create_err = buf;
    return code;
}

int cuda_fail(pss_system *s, cudaError_t e, const char *what) {
    return fail(s, e == cudaErrorMemoryAllocation ? PSS_ENOMEM : PSS_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call)                                                       \
    do {                                                               \
        cudaError_t _e = (call);                                       \
        if (_e != cudaSuccess) return cuda_fail(s, _e, #call);         \
    } while (0)

bool pow2_in(int n, int lo, int hi) { return n >= lo && n <= hi && (n & (n - 1)) == 0; }

size_t csize(const pss_system *s) { return s->prec == PSS_F64 ? 16 : 8; }
size_t rsize(const pss_system *s) { return s->prec == PSS_F64 ? 8 : 4; }
size_t fpsize(const pss_system *s) { return s->prec == PSS_F64 ? sizeof(FieldP<double>) : sizeof(FieldP<float>); }

// largest kept |k| on an axis of n points: (order+1)|k| < n; every |k| <= n/2
// is kept when order = 0
int kmax_axis(int n, int order) {
    if (n == 1) return 0;
    if (order <= 0) return n / 2;
    return std::min((n - 1) / (order + 1), n / 2);
}

// kept half-spectrum columns kx = 0..kmax (never more than the nx/2+1 stored)
int kept_cols(const pss_system *s, int fi) { return std::min(kmax_axis(s->nx, s->fields[fi].dealias) + 1, s->hx); }

template <typename T> SysP<T> sys_params(const pss_system *s) {
    SysP<T> p{};
    p.dim = s->dim;
    p.nx = s->nx; p.ny = s->ny; p.nz = s->nz; p.hx = s->hx;
    p.hxe = s->hx + (s->hx & 1);
    p.ntiles = s->ntiles; p.rows = s->rows;
    p.n_outer = s->n_outer; p.n_inner = s->n_inner;
    const double two_pi = 6.283185307179586476925286766559;
    p.gx = T(two_pi / (s->nx * s->dx[0]));
    p.gy = s->ny > 1 ? T(two_pi / (s->ny * s->dx[1])) : T(0);
    p.gz = s->nz > 1 ? T(two_pi / (s->nz * s->dx[2])) : T(0);
    p.dt = T(s->dt);
    p.inv_nsites = T(1.0 / (double)s->nsites);
    // programmatic dependent launch (tuning key "pdl"; by default only the
    // FFT-group kernels k2_col / k2_row take it, see pdl_fast)
    p.pdl = s->tune_pdl >= 0 ? s->tune_pdl : 0;
    p.wait_limit = s->tune_test_timeout ? kTestWaitLimit : 0;
    p.tx_extra = s->tune_test_timeout ? 16u : 0u;
    return p;
}

// Programmatic dependent launch of the FFT-group kernels, measured on GB300:
// the FP32 2D step gains (1024^2 15.7 -> 15.3, 512^2 11.4 -> 10.2, 256^2
// 7.8 -> 6.7 us/step; those kernels fetch their roots of unity and parameters
// before the wait), while the generic kernels lose (3D pair 360 -> 378 us,
// the adjoint's column kernels), so by default it is on for the former only.
int pdl_fast(const pss_system *s) { return s->tune_pdl >= 0 ? s->tune_pdl : 1; }

double pval(const pss_system *s, int inst, int id) {
    return id < 0 ? 1.0 : s->param_values[(size_t)inst * s->param_names.size() + id];
}

bool any_general(const pss_system *s) {
    for (const Field &f : s->fields)
        if (f.general) return true;
    return false;
}

bool same_mono(const std::vector<Mono> &a, const std::vector<Mono> &b) {
    if (a.size() != b.size()) return false;
    for (size_t i = 0; i < a.size(); ++i)
        if (a[i].param != b[i].param || a[i].scale != b[i].scale || a[i].pow != b[i].pow) return false;
    return true;
}

// The product terms of field fi (its power product, if any, among them),
// grouped by operator: a group's products add up in real space and take one
// transform.
std::vector<std::vector<GTerm>> term_groups(const pss_system *s, int fi) {
    std::vector<GTerm> terms;
    const Field &f = s->fields[fi];
    if (f.power > 0) terms.push_back({fi, f.rhs, {{fi, f.power, -1, 0}}});
    for (const GTerm &t : s->gterms)
        if (t.target == fi) terms.push_back(t);
    std::vector<std::vector<GTerm>> groups;
    for (const GTerm &t : terms) {
        bool placed = false;
        for (auto &g : groups)
            if (same_mono(g[0].M, t.M)) { g.push_back(t); placed = true; break; }
        if (!placed) groups.push_back({t});
    }
    return groups;
}

template <typename T> FieldP<T> field_params(const pss_system *s, int inst, int fi) {
    const Field &f = s->fields[fi];
    FieldP<T> p{};
    double O[kPolyTerms] = {0}, M[kPolyTerms] = {0};
    for (const Mono &m : f.lhs) O[m.pow] += m.scale * pval(s, inst, m.param);
    p.power = f.power;
    p.spectral = 0;
    if (f.general) {
        // one operator: the column kernel applies it after its own transform;
        // several: the products arrive summed in Fourier space with theirs
        const auto groups = term_groups(s, fi);
        p.power = 1;
        if (groups.size() == 1) {
            for (const Mono &m : groups[0][0].M) M[m.pow] += m.scale * pval(s, inst, m.param);
        } else {
            M[0] = 1.0;
            p.spectral = 1;
        }
    } else {
        for (const Mono &m : f.rhs) M[m.pow] += m.scale * pval(s, inst, m.param);
    }
    for (int i = 0; i < kPolyTerms; ++i) { p.O[i] = T(O[i]); p.M[i] = T(M[i]); }
    double dV = 1.0;
    for (int j = 0; j < s->dim; ++j) dV *= s->dx[j];
    p.noisy = f.noisy ? 1 : 0;
    p.sigma0 = f.noisy ? T(std::sqrt(std::max(0.0, (double)s->nsites * pval(s, inst, f.noise_param) * s->dt / dV)))
                       : T(0);
    p.noise_pow = f.noise_pow;
    p.kmax[0] = kmax_axis(s->nx, f.dealias);
    p.kmax[1] = kmax_axis(s->ny, f.dealias);
    p.kmax[2] = kmax_axis(s->nz, f.dealias);
    p.kx_cols = kept_cols(s, fi);
    p.field_id = fi;
    p.seed_lo = (uint32_t)(s->seeds[inst] & 0xffffffffu);
    p.seed_hi = (uint32_t)(s->seeds[inst] >> 32);
    return p;
}

// refresh the device copy of the per-slot parameters (ordered on the system's stream)
template <typename T> int upload_params_t(pss_system *s) {
    if (!s->fps_dirty) return PSS_OK;
    std::vector<FieldP<T>> h;
    h.reserve(s->nslots());
    for (int b = 0; b < s->batch; ++b)
        for (int fi = 0; fi < (int)s->fields.size(); ++fi) h.push_back(field_params<T>(s, b, fi));
    if (!h.empty()) CK(cudaMemcpyAsync(s->fps, h.data(), sizeof(FieldP<T>) * h.size(), cudaMemcpyHostToDevice, s->stream));
    s->fps_dirty = false;
    return PSS_OK;
}

int upload_params(pss_system *s) { return s->prec == PSS_F64 ? upload_params_t<double>(s) : upload_params_t<float>(s); }

// ---- launch shapes -------------------------------------------------------
// FFT radix cap of each kernel.  Radix 16 takes fewer passes (less shared-
// memory traffic and fewer barriers), radix 8 twice the threads per FFT
// (more warps to hide latency).  Measured on GB300: the column kernel is
// faster with radix 16 for 3D pencils and 1024-point columns, the row
// kernel with radix 8, the 3D y kernel with radix 16.
int col_emax(const pss_system *s) {
    if (s->tune_col_radix) return s->tune_col_radix;
    return (s->dim == 3 || s->n_inner >= 1024) ? 16 : 8;
}
int row_emax(const pss_system *s) { return s->tune_row_radix ? s->tune_row_radix : 8; }
int mid_emax(const pss_system *s) { return s->tune_mid_radix ? s->tune_mid_radix : 16; }

// tiles per CTA of the column kernel: a power of two, so that the CTA's
// FFT count F = tiles * kTileW * NP is one; aims at >= 64 threads per CTA
int col_tiles_per_cta(const pss_system *s) {
    const int NP = s->dim == 3 ? 2 : 1;
    const int per_tile = kTileW * NP * fft_TPF(s->n_inner, col_emax(s));
    if (s->tune_col_tiles > 0) {
        int tc = 1;
        while (tc * 2 <= s->tune_col_tiles && tc * 2 <= s->ntiles && 2 * tc * 2 * per_tile <= 512) tc *= 2;
        return tc;
    }
    int tc = 1;
    while (tc * 2 * per_tile <= 64 && tc * 2 <= s->ntiles) tc *= 2;
    return tc;
}

// row pairs per CTA of the row kernel: a power of two with G * TPF <= 128
// threads, and at least ~8 CTAs when there are few rows
int row_G(const pss_system *s) {
    const int tpf = fft_TPF(s->nx, row_emax(s));
    if (s->tune_row_pairs > 0) {
        int G = 1;
        while (G * 2 <= s->tune_row_pairs && G * 2 * tpf <= 256 && G * 2 <= std::max(1, s->rows / 2)) G *= 2;
        return G;
    }
    const int want = std::max(1, (s->rows / 2 + 7) / 8);
    int G = 1;
    while (G * 2 * tpf <= 128 && G * 2 <= want) G *= 2;
    return G;
}

int mid_PZ(const pss_system *s) {
    const int tpf = fft_TPF(s->ny, mid_emax(s));
    int pz = std::max(1, 256 / (kTileW * tpf));
    if (s->tune_mid_planes > 0) {
        int p = 1;
        while (p * 2 <= s->tune_mid_planes && p * 2 <= pz) p *= 2;
        pz = p;
    }
    pz = std::min(pz, s->nz);
    return pz;
}

// The FP32 2D path with one warp per transform serves sides of 256, 512 and
// 1024 points; everything else runs the generic kernels.

bool fast2d(const pss_system *s) {
    auto side = [](int n) { return n == 256 || n == 512 || n == 1024; };
    return s->tune_fast2d && s->prec == PSS_F32 && s->dim == 2 && side(s->nx) && side(s->ny) && !any_general(s);
}
// Launch shape of the fast path, measured on GB300.  2D: radix-16 passes for
// sides of 512 and 1024 (two warps per 1024-point transform, three passes),
// radix 8 for 256 (one warp per transform: the 256^2 step is latency-bound,
// 7.9 us against 9.7 us with radix 16), 4 row pairs per row CTA.  The 3D x
// pass takes radix 16 at every side: at 256 points that is half a warp per
// transform and two passes instead of three, and there the passes are bound
// by shared-memory bandwidth (x pass of the 256^3 pair 130 -> 113 us).
bool round_trip(const pss_system *s);

// A run of steps of a square FP32 2D system with one field and one instance
// on the FFT-group path is one persistent launch (k2p_step), where the
// device takes cooperative launches.
// The KPZ field of pss_add_grad_sq_term alone: one field whose explicit terms
// are M (d_x h)^2 + M (d_y h)^2 with one operator M (no power term).
bool kpz2d_shape(const pss_system *s) {
    if (s->dim != 2 || s->fields.size() != 1 || s->fields[0].power != 0 || s->gterms.size() != 2) return false;
    bool axis[2] = {false, false};
    for (const GTerm &t : s->gterms) {
        if (t.target != 0 || t.factors.size() != 1 || !same_mono(t.M, s->gterms[0].M)) return false;
        const GFactor &f = t.factors[0];
        if (f.field != 0 || f.power != 2 || f.lap != 0 || f.deriv < 0 || f.deriv > 1) return false;
        axis[f.deriv] = true;
    }
    return axis[0] && axis[1];
}
bool persist2d_ok(const pss_system *s) {
    auto side = [](int n) { return n == 256 || n == 512 || n == 1024; };
    if (!(s->tune_fast2d && s->prec == PSS_F32 && s->dim == 2 && side(s->nx) && s->nx == s->ny && s->batch == 1 &&
          s->fields.size() == 1 && s->coop && !round_trip(s) && (!any_general(s) || kpz2d_shape(s))))
        return false;
    // every CTA resident at once, and few enough column and row pairs per CTA
    // for its shared memory
    const int n = s->nx, uc = (n / 2 + 2) / 2;
    return std::max((uc + 1) / 2, n / 8) <= s->num_sms;
}
bool persist2d(const pss_system *s) { return s->tune_persist && persist2d_ok(s); }
int p2_mode(const pss_system *s) { return any_general(s) ? 1 : 0; }
// FFT pass radix of the persistent step: 16 at 1024 points (three passes of
// two warps per transform), 8 below (measured faster at 512: 6.2 against 8.3
// us per step)
int p2_radix(const pss_system *s) {
    const int r = s->tune_col2_radix ? s->tune_col2_radix : (s->ny >= 1024 ? 16 : 8);
    return r >= 16 ? 16 : 8;   // no radix-32 variant: it was slower than radix 16
}
// CTAs of the persistent step: every SM (one CTA each), but no more than the
// column pairs or row pairs to hand out, and at least enough to hold them (2
// column pairs and 4 row pairs per CTA)
int p2_blocks(const pss_system *s) {
    const int n = s->nx, uc = (n / 2 + 2) / 2;
    const int lo = std::max((uc + 1) / 2, n / 8);
    const int want = s->tune_persist_blocks > 0 ? s->tune_persist_blocks : std::min(s->num_sms, std::max(uc, n / 2));
    return std::min(s->num_sms, std::max(lo, want));
}

// Defaults of the FP32 2D two-kernel path.  A batch of 8 or more instances is
// throughput-bound rather than latency-bound; measured on GB300 (us per step,
// single-instance defaults -> batch defaults): 256^2 x 8 11.4 -> 9.5, x 32
// 36.4 -> 22.3, x 125 144 -> 77; 512^2 x 8 35.9 -> 25.3, x 32 130 -> 90,
// x 123 472 -> 325 (and 256^2 x 2 6.5 -> 8.0, hence the threshold).
bool big_batch(const pss_system *s) { return s->dim == 2 && s->batch >= 8 && s->nx <= 512; }
int col2_radix(const pss_system *s) {
    const int r = s->tune_col2_radix ? s->tune_col2_radix : ((s->ny >= 512 || big_batch(s)) ? 16 : 8);
    return r == 32 && s->ny != 1024 ? 16 : r;   // radix-32 passes serve 1024 points only
}
int row2_radix(const pss_system *s) {
    const int r = s->tune_row2_radix ? s->tune_row2_radix
                                     : ((s->dim == 3 || (s->nx >= 512 && !big_batch(s))) ? 16 : 8);
    return r == 32 && s->nx != 1024 ? 16 : r;
}
// CTA size limits of the two kernels (their launch bounds leave radix-32
// passes 128 registers per thread)
int col2_max_threads(int E) { return E == 8 ? 1024 : E == 16 ? 768 : 512; }
int row2_max_threads(int E) { return E == 32 ? 512 : 1024; }
int col2_warps(const pss_system *s) {
    const int E = col2_radix(s);
    const int fft_warps = 4 * s->ny / E / 32;
    const int want = s->tune_col2_warps > 0 ? s->tune_col2_warps : (big_batch(s) && s->ny == 256 ? 4 : 8);
    return std::max(1, std::min(want, col2_max_threads(E) / 32 - fft_warps));
}
int row2_noise_warps(const pss_system *s, int pairs) {
    const int E = row2_radix(s);
    const int fft_warps = pairs * s->nx / E / 32;
    const int want = s->tune_row2_noise > 0 ? s->tune_row2_noise : (big_batch(s) && s->nx == 256 ? 8 : 16);
    return std::max(1, std::min(want, row2_max_threads(E) / 32 - fft_warps));
}
bool any_noisy(const pss_system *s) {
    for (const Field &f : s->fields)
        if (f.noisy) return true;
    return false;
}
// row pairs per CTA: a power of two with at most 512 threads per CTA
int row2_pairs(const pss_system *s) {
    const int tpf = s->nx / row2_radix(s);
    const int nw = s->tune_row2_pairs > 0 ? s->tune_row2_pairs : (big_batch(s) ? 8 : 4);
    int p = 1;
    while (p * tpf < 32) p *= 2;   // whole warps of transform threads
    while (p * 2 <= nw && p * 2 <= 8 && p * 2 * tpf <= 512) p *= 2;
    return p;
}

// row pairs per CTA of the adjoint's x pass on FFT groups.  It has no noise
// warps, so a CTA is just its transform groups: the pairs are spread so that
// every SM gets a CTA (at 256^2 the step's 4 pairs would leave 32 CTAs of
// four warps on 152 SMs), with whole warps of transform threads.
int row2_adj_pairs(const pss_system *s, int nslots) {
    const int tpf = s->nx / row2_radix(s);
    const int maxp = std::min(8, row2_max_threads(row2_radix(s)) / tpf);
    int p = 1;
    while (p * tpf < 32) p *= 2;
    if (s->tune_adj_row_pairs > 0) {
        while (p * 2 <= s->tune_adj_row_pairs && p * 2 <= maxp) p *= 2;
        return p;
    }
    while (p * 2 <= maxp && (long long)s->rows / (4 * p) * nslots >= s->num_sms) p *= 2;
    return p;
}

// The FP32 3D step runs its x pass (rows of 256, 512 or 1024 points) with
// the FFT groups of the fast path, on the tiled arrays of the generic kernels.
bool fast3d_rows(const pss_system *s) {
    return s->tune_fast3d && s->prec == PSS_F32 && s->dim == 3 && (s->nx == 256 || s->nx == 512 || s->nx == 1024);
}

int max_kept_tiles(const pss_system *s) {
    int m = 0;
    for (int i = 0; i < (int)s->fields.size(); ++i) m = std::max(m, (kept_cols(s, i) + kTileW - 1) / kTileW);
    return std::min(m, s->ntiles);
}

// Optional per-launch CUDA events (pss_time_kernels): kind 0 = k_col,
// 1 = k_mid inverse, 2 = k_row, 3 = k_mid forward.  The events are recorded
// into a captured graph as event-record nodes, so that the GPU never waits
// for the host between an event and its kernel.
struct Timer {
    std::vector<cudaEvent_t> ev[4];
    int begin(int kind, cudaStream_t st) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return -1;
        ev[kind].push_back(e);
        return cudaEventRecordWithFlags(e, st, cudaEventRecordExternal) == cudaSuccess ? 0 : -1;
    }
    ~Timer() {
        for (auto &v : ev)
            for (cudaEvent_t e : v) cudaEventDestroy(e);
    }
};

// ---- kernel sequences ----------------------------------------------------
// A sequence acts on slots slot0 .. slot0 + nslots - 1.  real_stride = 0 makes
// every slot of a real-space transfer use the same (one-slot) scratch.
template <typename T> struct Seq {
    pss_system *s;
    cudaStream_t st;
    int slot0, nslots;
    Timer *timer = nullptr;
    // a product-term factor in flight: the column inverse applies op(q), the
    // row inverse folds r^n into the term's product instead of storing r
    int op_on = 0, op_deriv = -1, op_lap = 0;
    T *fac_acc = nullptr, *fac_tp = nullptr;
    int fac_power = 1, fac_first_factor = 1, fac_last_factor = 1, fac_first_term = 1;

    cplx<T> *state() const { return (cplx<T> *)s->state; }
    cplx<T> *A() const { return (cplx<T> *)s->A; }
    cplx<T> *B() const { return (cplx<T> *)s->B; }

    int col(int mode, bool in_is_B, bool out_is_A) {
        return col_ptrs(mode, state(), in_is_B ? B() : A(), out_is_A ? A() : B(), nullptr, 0);
    }

    int col_ptrs(int mode, cplx<T> *st_ptr, const cplx<T> *in_ptr, cplx<T> *out_ptr, const cplx<T> *aux,
                 long long adj_step, cplx<T> *st_out = nullptr, const cplx<T> *in2 = nullptr) {
        ColArgs<T> a{};
        a.sp = sys_params<T>(s);
        a.fps = (const FieldP<T> *)s->fps;
        a.in = in_ptr;
        a.out = out_ptr;
        a.state = st_ptr;
        a.state_out = st_out;
        a.aux = aux;
        a.adj_step = adj_step;
        a.d_adj_base = (mode == COL_ADJ_A || mode == COL_ADJ_B || mode == COL_ADJ_BA) ? s->d_seg + 1 : nullptr;
        a.grad = s->d_grad;
        a.in_colmajor = (mode == COL_ADJ_A && fast2d(s)) ? 1 : 0;   // the product the fast path recomputed
        a.in2 = in2;
        a.in2_colmajor = fast2d(s) ? 1 : 0;
        a.op_on = op_on;
        a.op_deriv = op_deriv;
        a.op_lap = op_lap;
        a.slot_stride = s->field_elems;
        a.slot0 = slot0;
        a.tw = (const cplx<T> *)s->tw;
        a.d_step = s->d_step;
        a.d_status = s->d_status;
        a.mode = mode;
        a.E = col_emax(s);
        a.tiles_per_cta = col_tiles_per_cta(s);
        a.F = a.tiles_per_cta * kTileW * (s->dim == 3 ? 2 : 1);
        a.n_tiles = mode == COL_INV_MASK ? max_kept_tiles(s) : s->ntiles;
        const int gx = (a.n_tiles + a.tiles_per_cta - 1) / a.tiles_per_cta;
        const int gy = s->dim == 3 ? s->ny / 2 + 1 : 1;
        if constexpr (std::is_same<T, float>::value) {
            // the adjoint's column part of the FP32 2D path on FFT groups: one
            // column pair per CTA
            if ((mode == COL_ADJ_A || mode == COL_ADJ_B || mode == COL_ADJ_BA) && fast2d(s) && s->tune_adj_col2) {
                a.E = col2_radix(s) == 16 ? 16 : 8;
                if (timer) timer->begin(0, st);
                cudaError_t e = launch_col2_adj(a, nslots, st);
                if (timer) timer->begin(0, st);
                s->launches++;
                if (e != cudaSuccess) return cuda_fail(s, e, "k2_col_adj launch");
                return PSS_OK;
            }
        }
        if (timer) timer->begin(0, st);
        cudaError_t e = launch_col<T>(a, nslots, gx, gy, st);
        if (timer) timer->begin(0, st);
        s->launches++;
        if (e != cudaSuccess) return cuda_fail(s, e, "k_col launch");
        return PSS_OK;
    }

    // in: A or B (complex), or real (ROW_R2C); out: A or B (complex), or real (ROW_C2R)
    int row(int mode, bool in_is_A, bool out_is_B, bool inc, void *real, size_t real_stride) {
        return row_ptrs(mode, in_is_A ? A() : B(), out_is_B ? B() : A(), inc, (const T *)real, (T *)real, real_stride);
    }

    int row_ptrs(int mode, const cplx<T> *in_ptr, cplx<T> *out_ptr, bool inc, const T *real_in, T *real_out,
                 size_t real_stride) {
        RowArgs<T> a{};
        a.sp = sys_params<T>(s);
        a.fps = (const FieldP<T> *)s->fps;
        a.in = in_ptr;
        a.out = out_ptr;
        a.real_in = real_in;
        a.real_out = real_out;
        a.slot_stride = s->field_elems;
        a.real_stride = real_stride;
        a.slot0 = slot0;
        a.tw = (const cplx<T> *)s->tw;
        a.d_step = s->d_step;
        a.d_status = s->d_status;
        a.mode = mode;
        a.E = row_emax(s);
        a.G = row_G(s);
        a.kx_cols_max = 0;
        for (int i = 0; i < (int)s->fields.size(); ++i) a.kx_cols_max = std::max(a.kx_cols_max, kept_cols(s, i));
        a.inc_step = inc ? 1 : 0;
        a.fac_acc = fac_acc;
        a.fac_tp = fac_tp;
        a.fac_power = fac_power;
        a.fac_first_factor = fac_first_factor;
        a.fac_last_factor = fac_last_factor;
        a.fac_first_term = fac_first_term;
        if (timer) timer->begin(2, st);
        cudaError_t e = launch_row<T>(a, nslots, st);
        if (timer) timer->begin(2, st);
        s->launches++;
        if (e != cudaSuccess) return cuda_fail(s, e, "k_row launch");
        return PSS_OK;
    }

    int mid(int mode, bool in_is_A, bool inc) { return mid_ptrs(mode, in_is_A ? A() : B(), in_is_A ? B() : A(), inc); }

    int mid_ptrs(int mode, const cplx<T> *in_ptr, cplx<T> *out_ptr, bool inc) {
        MidArgs<T> a{};
        a.sp = sys_params<T>(s);
        a.fps = (const FieldP<T> *)s->fps;
        a.in = in_ptr;
        a.out = out_ptr;
        a.slot_stride = s->field_elems;
        a.slot0 = slot0;
        a.tw = (const cplx<T> *)s->tw;
        a.d_step = s->d_step;
        a.d_status = s->d_status;
        a.mode = mode;
        a.E = mid_emax(s);
        a.PZ = mid_PZ(s);
        a.inc_step = inc ? 1 : 0;
        const int nt = mode == MID_INV_MASK ? max_kept_tiles(s) : s->ntiles;
        const int kind = mode == MID_FWD ? 3 : 1;
        if (timer) timer->begin(kind, st);
        cudaError_t e = launch_mid<T>(a, nslots, nt, st);
        if (timer) timer->begin(kind, st);
        s->launches++;
        if (e != cudaSuccess) return cuda_fail(s, e, "k_mid launch");
        return PSS_OK;
    }

    // the fast 2D path (FP32 only): k2_col, then k2_row
    int col2(int mode) { return col2_ptrs(mode, state(), B(), A(), nullptr); }

    int col2_ptrs(int mode, cplx<T> *st_ptr, const cplx<T> *in_ptr, cplx<T> *out_ptr, cplx<T> *st_out) {
        if constexpr (std::is_same<T, float>::value) {
            ColArgs<float> a{};
            a.sp = sys_params<float>(s);
            a.sp.pdl = pdl_fast(s);
            a.fps = (const FieldP<float> *)s->fps;
            a.in = in_ptr;
            a.out = out_ptr;
            a.state = st_ptr;
            a.state_out = st_out;
            a.slot_stride = s->field_elems;
            a.slot0 = slot0;
            a.tw = (const float2 *)s->tw;
            a.d_step = s->d_step;
            a.d_status = s->d_status;
            a.mode = mode;
            a.aux_warps = col2_warps(s);
            a.E = col2_radix(s);
            a.noise = any_noisy(s) ? (const float2 *)s->XI : nullptr;
            const int nt = mode == COL_INV_MASK ? max_kept_tiles(s) : s->ntiles;
            if (timer) timer->begin(0, st);
            cudaError_t e = launch_col2(a, nslots, nt, st);
            if (timer) timer->begin(0, st);
            s->launches++;
            if (e != cudaSuccess) return cuda_fail(s, e, "k2_col launch");
            return PSS_OK;
        } else {
            (void)mode; (void)st_ptr; (void)in_ptr; (void)out_ptr; (void)st_out;
            return fail(s, PSS_EUNSUPPORTED, "the FFT-group 2D path is FP32 only");
        }
    }

    // (the step counter is advanced by k2_col; inc documents the caller's intent)
    int row2(bool inc) { (void)inc; return row2_ptrs(A(), B(), nullptr); }

    int row2_ptrs(const cplx<T> *in_ptr, cplx<T> *out_ptr, T *real_out) {
        if constexpr (std::is_same<T, float>::value) {
            RowArgs<float> a{};
            a.sp = sys_params<float>(s);
            a.sp.pdl = pdl_fast(s);
            a.fps = (const FieldP<float> *)s->fps;
            a.in = in_ptr;
            a.out = out_ptr;
            a.real_out = real_out;
            a.real_stride = 0;   // one slot (the adjoint's recompute)
            a.slot_stride = s->field_elems;
            a.slot0 = slot0;
            a.tw = (const float2 *)s->tw;
            a.d_step = s->d_step;
            a.d_status = s->d_status;
            a.mode = ROW_FUSED;
            a.G = row2_pairs(s);
            a.E = row2_radix(s);
            a.kx_cols_max = 0;
            for (int i = 0; i < (int)s->fields.size(); ++i) a.kx_cols_max = std::max(a.kx_cols_max, kept_cols(s, i));
            a.inc_step = 0;   // k2_col advances the step counter
            a.noise = any_noisy(s) ? (float2 *)s->XI : nullptr;
            a.noise_warps = a.noise ? row2_noise_warps(s, a.G) : 0;
            // optionally, SMs the row CTAs leave idle draw part of the noise in
            // extra CTAs (measured at 1024^2: slower than spreading the noise
            // over the row CTAs, 19.0 against 16.0 us/step at 75 %, so off by default)
            const int row_ctas = s->rows / (2 * a.G) * nslots;
            const int share = s->tune_row2_share >= 0 ? s->tune_row2_share : 0;
            a.noise_ctas = (a.noise && share > 0 && nslots == 1) ? std::max(0, s->num_sms - row_ctas) : 0;
            a.noise_share = a.noise_ctas > 0 ? std::min(64, share * 64 / 100) : 0;
            if (timer) timer->begin(2, st);
            cudaError_t e = launch_row2(a, nslots, st, false);
            if (timer) timer->begin(2, st);
            s->launches++;
            if (e != cudaSuccess) return cuda_fail(s, e, "k2_row launch");
            return PSS_OK;
        } else {
            (void)in_ptr; (void)out_ptr; (void)real_out;
            return fail(s, PSS_EUNSUPPORTED, "the FFT-group 2D path is FP32 only");
        }
    }

    // the 3D x pass with FFT groups (FP32): B -> A, tiled arrays
    int row3() {
        if constexpr (std::is_same<T, float>::value) {
            RowArgs<float> a{};
            a.sp = sys_params<float>(s);
            a.fps = (const FieldP<float> *)s->fps;
            a.in = B();
            a.out = A();
            a.slot_stride = s->field_elems;
            a.slot0 = slot0;
            a.tw = (const float2 *)s->tw;
            a.d_step = s->d_step;
            a.d_status = s->d_status;
            a.mode = ROW_FUSED;
            a.E = row2_radix(s);
            a.G = std::min(8, 256 / (s->nx / a.E));   // row pairs per CTA: 256 threads
            a.kx_cols_max = 0;
            for (int i = 0; i < (int)s->fields.size(); ++i) a.kx_cols_max = std::max(a.kx_cols_max, kept_cols(s, i));
            a.inc_step = 0;
            a.noise = nullptr;
            a.noise_warps = 0;
            if (timer) timer->begin(2, st);
            cudaError_t e = launch_row2(a, nslots, st, true);
            if (timer) timer->begin(2, st);
            s->launches++;
            if (e != cudaSuccess) return cuda_fail(s, e, "k2_row (3D x pass) launch");
            return PSS_OK;
        } else {
            return fail(s, PSS_EUNSUPPORTED, "the FFT-group x pass is FP32 only");
        }
    }

    // the 2D adjoint's x pass on FFT groups (FP32): A -> B (tiled), times p r^(p-1)
    int row2_adj(const T *real_r) {
        if constexpr (std::is_same<T, float>::value) {
            RowArgs<float> a{};
            a.sp = sys_params<float>(s);
            a.fps = (const FieldP<float> *)s->fps;
            a.in = A();
            a.out = B();
            a.real_in = real_r;
            a.real_stride = 0;
            a.slot_stride = s->field_elems;
            a.slot0 = slot0;
            a.tw = (const float2 *)s->tw;
            a.d_step = s->d_step;
            a.d_status = s->d_status;
            a.mode = ROW_ADJ;
            a.E = row2_radix(s);
            a.G = row2_adj_pairs(s, nslots);
            a.kx_cols_max = s->hx;
            if (timer) timer->begin(2, st);
            cudaError_t e = launch_row2(a, nslots, st, true);
            if (timer) timer->begin(2, st);
            s->launches++;
            if (e != cudaSuccess) return cuda_fail(s, e, "k2_row (adjoint x pass) launch");
            return PSS_OK;
        } else {
            (void)real_r;
            return fail(s, PSS_EUNSUPPORTED, "the FFT-group x pass is FP32 only");
        }
    }

    int x_pass_3d() { return fast3d_rows(s) ? row3() : row(ROW_FUSED, false, false, false, nullptr, 0); }  // B -> A

    // The explicit part of general field fi of instance inst, for the
    // sequence's one slot (section "Writing models": N = M prod_k psi_k^n_k,
    // psi_k a field acted on by a differential operator): every factor goes
    // to real space from op(q) m phi of its field, the factors multiply and
    // the terms of a group (one operator M) add up there; the sum goes back
    // along x (and y in 3D) into B, where the column kernel transforms it
    // the rest of the way and applies M.  With several groups each sum is
    // transformed completely and B takes sum_g M_g(q) F[sum_g] instead.
    // Replaces what the fused kernels wrote into B for this slot.
    int general_product(int inst, int fi) {
        int rc;
        cudaError_t e;
        const int nf = (int)s->fields.size();
        const auto groups = term_groups(s, fi);
        const bool spectral = groups.size() > 1;
        const size_t stride = s->field_elems;
        cplx<T> *G = (cplx<T> *)s->GS;
        T *acc = (T *)s->real_acc, *tp = (T *)s->real_tp;
        for (size_t gi = 0; gi < groups.size(); ++gi) {
            const auto &g = groups[gi];
            for (size_t ti = 0; ti < g.size(); ++ti) {
                const auto &fac = g[ti].factors;
                for (size_t k = 0; k < fac.size(); ++k) {
                    // the factor's field (same instance), kept modes times op(q), to
                    // real space; its own slot of A (and of G in 3D) is scratch
                    Seq<T> q{s, st, inst * nf + fac[k].field, 1};
                    q.op_on = 1;
                    q.op_deriv = fac[k].deriv;
                    q.op_lap = fac[k].lap;
                    q.fac_acc = acc;
                    q.fac_tp = tp;
                    q.fac_power = fac[k].power;
                    q.fac_first_factor = k == 0;
                    q.fac_last_factor = k + 1 == fac.size();
                    q.fac_first_term = ti == 0;
                    if ((rc = q.col_ptrs(COL_INV_MASK, q.state(), nullptr, q.A(), nullptr, 0))) return rc;   // -> A
                    if (s->dim == 3) {
                        if ((rc = q.mid_ptrs(MID_INV_MASK, q.A(), G, false))) return rc;                   // A -> G
                        if ((rc = q.row_ptrs(ROW_C2R_KEPT, G, q.A(), false, nullptr, nullptr, 0))) return rc;
                    } else if ((rc = q.row_ptrs(ROW_C2R_KEPT, q.A(), q.B(), false, nullptr, nullptr, 0))) {
                        return rc;
                    }
                }
            }
            if (!spectral) {
                if (s->dim == 3) {
                    if ((rc = row_ptrs(ROW_R2C, A(), A(), false, acc, nullptr, 0))) return rc;   // -> A
                    return mid_ptrs(MID_FWD, A(), B(), false);                                 // A -> B
                }
                return row_ptrs(ROW_R2C, A(), B(), false, acc, nullptr, 0);                      // -> B
            }
            // the group's sum transformed along every axis, times M_g, into B
            cplx<T> *full;
            if ((rc = row_ptrs(ROW_R2C, A(), A(), false, acc, nullptr, 0))) return rc;           // -> A
            if (s->dim == 3) {
                if ((rc = mid_ptrs(MID_FWD, A(), G, false))) return rc;                         // A -> G
                if ((rc = col_ptrs(COL_FWD, A(), G, B(), nullptr, 0))) return rc;                // G -> A
                full = A();
            } else {
                if ((rc = col_ptrs(COL_FWD, G, A(), B(), nullptr, 0))) return rc;                // A -> G
                full = G;
            }
            double m[kPolyTerms] = {0};
            for (const Mono &mo : g[0].M) m[mo.pow] += mo.scale * pval(s, inst, mo.param);
            e = launch_combine<T>(sys_params<T>(s), B() + (size_t)slot0 * stride, full + (size_t)slot0 * stride, m,
                                  gi == 0, st);
            s->launches++;
            if (e != cudaSuccess) return cuda_fail(s, e, "combine kernel");
        }
        return PSS_OK;
    }

    // B <- x-transformed product of the current state (start of a run)
    int prologue() {
        int rc;
        if (fast2d(s)) {
            if ((rc = col2(COL_INV_MASK))) return rc;                             // state -> A (column-major)
            return row2(false);                                                    // A -> B (column-major)
        }
        if ((rc = col(COL_INV_MASK, false, true))) return rc;                      // state -> A
        if (s->dim == 3) {
            if ((rc = mid(MID_INV_MASK, true, false))) return rc;                  // A -> B
            if ((rc = x_pass_3d())) return rc;                                     // B -> A
            return mid(MID_FWD, true, false);                                      // A -> B
        }
        return row(ROW_FUSED, true, true, false, nullptr, 0);                       // A -> B
    }

    int one_step() {
        int rc;
        if (fast2d(s)) {
            if ((rc = col2(COL_STEP))) return rc;                                 // B, state -> state, A
            return row2(true);                                                     // A -> B, step++
        }
        if ((rc = col(COL_STEP, true, true))) return rc;                           // B, state -> state, A
        if (s->dim == 3) {
            if ((rc = mid(MID_INV_MASK, true, false))) return rc;                  // A -> B
            if ((rc = x_pass_3d())) return rc;                                     // B -> A
            return mid(MID_FWD, true, true);                                       // A -> B, step++
        }
        return row(ROW_FUSED, true, true, true, nullptr, 0);                        // A -> B, step++
    }

    // real scratch -> state of the sequence's slots
    int forward_from_real() {
        int rc;
        if (s->dim == 3) {
            if ((rc = row(ROW_R2C, true, false, false, s->real, 0))) return rc;   // real -> A
            if ((rc = mid(MID_FWD, true, false))) return rc;                      // A -> B
        } else {
            if ((rc = row(ROW_R2C, true, true, false, s->real, 0))) return rc;    // real -> B
        }
        return col(COL_FWD, true, true);                                          // B -> state
    }

    // state -> real scratch
    int inverse_to_real() {
        int rc;
        if ((rc = col(COL_INV_FULL, false, true))) return rc;                     // state -> A
        if (s->dim == 3) {
            if ((rc = mid(MID_INV_FULL, true, false))) return rc;                 // A -> B
            return row(ROW_C2R, false, false, false, s->real, 0);                 // B -> real
        }
        return row(ROW_C2R, true, false, false, s->real, 0);                      // A -> real
    }

    // Recompute of one forward step for the adjoint: phi_n (st_in) -> phi_n+1
    // (st_out), reading the x(y)-transformed product of phi_n (prod_in) and
    // writing that of phi_n+1 (prod_out) and the de-aliased real field
    // r_n+1 = F^-1[m phi_n+1] (real_out), which the adjoint step needs.
    int recompute_step(cplx<T> *st_in, cplx<T> *st_out, const cplx<T> *prod_in, cplx<T> *prod_out, T *real_out) {
        int rc;
        if (fast2d(s)) {   // the kernels (and the column-major product) of the forward run
            if ((rc = col2_ptrs(COL_STEP, st_in, prod_in, A(), st_out))) return rc;          // -> A, step++
            return row2_ptrs(A(), prod_out, real_out);                                       // A -> prod, r, noise
        }
        if ((rc = col_ptrs(COL_STEP, st_in, prod_in, A(), nullptr, 0, st_out))) return rc;  // -> A
        if (s->dim == 3) {
            if ((rc = mid(MID_INV_MASK, true, false))) return rc;                            // A -> B
            if ((rc = row_ptrs(ROW_FUSED, B(), A(), false, nullptr, real_out, 0))) return rc; // B -> A, r
            return mid_ptrs(MID_FWD, A(), prod_out, true);                                   // A -> prod, step++
        }
        return row_ptrs(ROW_FUSED, A(), prod_out, true, nullptr, real_out, 0);               // A -> prod, r, step++
    }

    // The product and real field of the state st (start of a recomputed segment).
    int recompute_prologue(cplx<T> *st, cplx<T> *prod_out, T *real_out) {
        int rc;
        if (fast2d(s)) {
            if ((rc = col2_ptrs(COL_INV_MASK, st, nullptr, A(), nullptr))) return rc;         // st -> A
            return row2_ptrs(A(), prod_out, real_out);                                       // A -> prod, r, noise
        }
        if ((rc = col_ptrs(COL_INV_MASK, st, nullptr, A(), nullptr, 0))) return rc;           // st -> A
        if (s->dim == 3) {
            if ((rc = mid(MID_INV_MASK, true, false))) return rc;                            // A -> B
            if ((rc = row_ptrs(ROW_FUSED, B(), A(), false, nullptr, real_out, 0))) return rc; // B -> A, r
            return mid_ptrs(MID_FWD, A(), prod_out, false);                                  // A -> prod
        }
        return row_ptrs(ROW_FUSED, A(), prod_out, false, nullptr, real_out, 0);              // A -> prod, r
    }

    // One adjoint step for the forward step phi_n -> phi_n1 (noise step n_step),
    // with s->L holding lambda_{n+1} on entry, lambda_n on exit; prod is the
    // x(y)-transformed product of phi_n and real_r its de-aliased real field
    // (see the adjoint recursion in COL_ADJ_A / COL_ADJ_B).
    //   part A: mu = g lambda, gradients, nu = dt M mu back along the slowest axis -> A
    //   x(y) part: w = p r^(p-1) N F^-1[nu] in real space, then its x(y) transform -> B
    //   part B: lambda_n = mu + m F[w] / N
    // Over a run of steps, part B of one step and part A of the step before it
    // share one launch (COL_ADJ_BA) where its shared memory fits.
    bool fused_adjoint() const {
        const int F = col_tiles_per_cta(s) * kTileW * (s->dim == 3 ? 2 : 1);
        const size_t need = col_smem_bytes<T>(s->n_inner, F, col_emax(s), COL_ADJ_BA);
        return s->tune_fuse_adj && need > 0 && need <= 227 * 1024;
    }

    int adjoint_part_a(const cplx<T> *phi_n1, const cplx<T> *prod, long long n_step) {
        return col_ptrs(COL_ADJ_A, (cplx<T> *)s->L, prod, A(), phi_n1, n_step);
    }

    int adjoint_part_b(long long n_step) { return col_ptrs(COL_ADJ_B, (cplx<T> *)s->L, B(), A(), nullptr, n_step); }

    // part B of step n, then part A of step n - 1 (phi_n, prod_{n-1}, noise step n - 1)
    int adjoint_part_ba(const cplx<T> *phi_n, const cplx<T> *prod_prev, long long n_step) {
        return col_ptrs(COL_ADJ_BA, (cplx<T> *)s->L, B(), A(), phi_n, n_step - 1, nullptr, prod_prev);
    }

    int adjoint_x_part(const T *real_r) {
        int rc;
        if (s->dim == 3) {
            if ((rc = mid(MID_INV_FULL, true, false))) return rc;                            // A -> B
            if ((rc = row_ptrs(ROW_ADJ, B(), A(), false, real_r, nullptr, 0))) return rc;     // B -> A
            if ((rc = mid(MID_FWD, true, false))) return rc;                                 // A -> B
        } else if (fast2d(s)) {
            if ((rc = row2_adj(real_r))) return rc;                                          // A -> B
        } else {
            if ((rc = row_ptrs(ROW_ADJ, A(), B(), false, real_r, nullptr, 0))) return rc;     // A -> B
        }
        return PSS_OK;
    }

    int adjoint_step(const cplx<T> *phi_n1, const cplx<T> *prod, const T *real_r, long long n_step) {
        int rc;
        if ((rc = adjoint_part_a(phi_n1, prod, n_step))) return rc;
        if ((rc = adjoint_x_part(real_r))) return rc;
        return adjoint_part_b(n_step);
    }
};

// the products of the general fields' slots, over what the fused kernels wrote
template <typename T> int general_products(pss_system *s, cudaStream_t st) {
    const int nf = (int)s->fields.size();
    for (int slot = 0; slot < s->nslots(); ++slot)
        if (s->fields[slot % nf].general) {
            int rc = Seq<T>{s, st, slot, 1}.general_product(slot / nf, slot % nf);
            if (rc) return rc;
        }
    return PSS_OK;
}

template <typename T> int full_prologue(pss_system *s, cudaStream_t st) {
    int rc = Seq<T>{s, st, 0, s->nslots()}.prologue();
    if (rc || !any_general(s)) return rc;
    return general_products<T>(s, st);
}

template <typename T> int run_prologue(pss_system *s) { return full_prologue<T>(s, s->stream); }

int alloc_term_scratch(pss_system *s) {
    if (!any_general(s)) return PSS_OK;
    if (!s->GS) CK(cudaMalloc(&s->GS, csize(s) * s->field_elems * (size_t)s->nslots()));
    if (!s->real) CK(cudaMalloc(&s->real, rsize(s) * (size_t)s->nsites));
    if (!s->real_acc) CK(cudaMalloc(&s->real_acc, rsize(s) * (size_t)s->nsites));
    if (!s->real_tp) CK(cudaMalloc(&s->real_tp, rsize(s) * (size_t)s->nsites));
    return PSS_OK;
}

// Makes B hold the product of the current state (and, on the FP32 2D path, XI
// the current step's noise) for the step kernels.  With for_persist the run
// that follows is a persistent launch, which computes both itself when they
// are stale (its prologue flag): only the arrays are allocated here.
int prologue(pss_system *s, bool for_persist = false) {
    if (int rc = alloc_term_scratch(s)) return rc;
    if (for_persist) {
        if (!s->XI) {
            const size_t bytes = csize(s) * s->field_elems * (size_t)s->nslots();
            CK(cudaMalloc(&s->XI, bytes));
            CK(cudaMemset(s->XI, 0, bytes));
        }
        return PSS_OK;
    }
    if (!s->stale && s->b_fast == fast2d(s)) return PSS_OK;
    if (fast2d(s) && !s->XI) {
        const size_t bytes = csize(s) * s->field_elems * (size_t)s->nslots();
        CK(cudaMalloc(&s->XI, bytes));
        CK(cudaMemset(s->XI, 0, bytes));
    }
    int rc = s->prec == PSS_F64 ? run_prologue<double>(s) : run_prologue<float>(s);
    if (rc) return rc;
    s->stale = false;
    s->b_fast = fast2d(s);
    return PSS_OK;
}

// Every step ends in real space when a field has a boundary frame (section
// "Callback functions": the frame is set on the real field at the end of a
// step) or when the round trip is asked for as an ablation.
bool round_trip(const pss_system *s) {
    if (s->tune_real_state) return true;
    for (const Field &f : s->fields)
        if (f.frame_w > 0) return true;
    return false;
}

template <typename T> int step_once(pss_system *s, cudaStream_t st) {
    int rc = Seq<T>{s, st, 0, s->nslots()}.one_step();
    if (rc) return rc;
    if (!round_trip(s)) return any_general(s) ? general_products<T>(s, st) : PSS_OK;
    // per slot: the full real field, its frame, and back to the spectrum
    const int nf = (int)s->fields.size();
    for (int slot = 0; slot < s->nslots(); ++slot) {
        Seq<T> q{s, st, slot, 1};
        if ((rc = q.inverse_to_real())) return rc;
        const Field &f = s->fields[slot % nf];
        if (f.frame_w > 0) {
            cudaError_t e = launch_frame<T>((T *)s->real, s->nx, (long long)s->ny * s->nz, f.frame_w, f.frame_lo,
                                            f.frame_hi, st);
            s->launches++;
            if (e != cudaSuccess) return cuda_fail(s, e, "frame kernel");
        }
        if ((rc = q.forward_from_real())) return rc;
    }
    // the product (and on the FP32 2D path the noise) of the new state
    return full_prologue<T>(s, st);
}

int record_steps(pss_system *s, cudaStream_t st, int64_t n) {
    for (int64_t k = 0; k < n; ++k) {
        int rc = s->prec == PSS_F64 ? step_once<double>(s, st) : step_once<float>(s, st);
        if (rc) return rc;
    }
    return PSS_OK;
}

// capture `steps` steps of every system into one graph (on systems[0]'s
// capture stream).  Distinct systems share no buffers, so each one's steps
// form a branch of its own (forked from and joined to the capture stream by
// events, recorded on the system's own capture stream) and the GPU runs the
// branches side by side; a system listed twice keeps the serial order.
int capture_graph(pss_system **sys, int n, int steps, cudaGraphExec_t *out) {
    pss_system *s = sys[0];
    bool branches = n > 1;
    for (int i = 0; i < n && branches; ++i)
        for (int j = 0; j < i; ++j)
            if (sys[i] == sys[j] || sys[i]->cap_stream == sys[j]->cap_stream) branches = false;
    std::vector<cudaEvent_t> ev(branches ? n + 1 : 0, nullptr);
    for (auto &x : ev) {
        cudaError_t e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            for (auto &y : ev) if (y) cudaEventDestroy(y);
            return cuda_fail(s, e, "cudaEventCreateWithFlags");
        }
    }
    auto destroy_events = [&]() { for (auto &x : ev) if (x) cudaEventDestroy(x); };
    cudaError_t e = cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { destroy_events(); return cuda_fail(s, e, "cudaStreamBeginCapture"); }
    int rc = PSS_OK;
    std::vector<int64_t> before(n);
    for (int i = 0; i < n; ++i) before[i] = sys[i]->launches;
    if (branches) {
        e = cudaEventRecord(ev[n], s->cap_stream);                               // fork
        int forked = 1;
        for (; forked < n && e == cudaSuccess; ++forked) e = cudaStreamWaitEvent(sys[forked]->cap_stream, ev[n], 0);
        if (e != cudaSuccess) { rc = cuda_fail(s, e, "forking the capture"); --forked; }
        for (int i = 0; i < n && rc == PSS_OK; ++i) {
            rc = record_steps(sys[i], sys[i]->cap_stream, steps);
            if (rc && i != 0) s->err = sys[i]->err;
        }
        // join every forked stream, also after a failure, so that the capture ends cleanly
        for (int i = 1; i < forked; ++i) {
            e = cudaEventRecord(ev[i], sys[i]->cap_stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s->cap_stream, ev[i], 0);
            if (e != cudaSuccess && rc == PSS_OK) rc = cuda_fail(s, e, "joining the capture");
        }
    } else {
        for (int k = 0; k < steps && rc == PSS_OK; ++k)
            for (int i = 0; i < n && rc == PSS_OK; ++i) {
                rc = record_steps(sys[i], s->cap_stream, 1);
                if (rc && i != 0) s->err = sys[i]->err;
            }
    }
    for (int i = 0; i < n; ++i) {
        sys[i]->graph_launches = steps > 0 ? (sys[i]->launches - before[i]) / steps : 0;
        sys[i]->launches = before[i];
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s->cap_stream, &g);
    destroy_events();
    if (rc) { if (g) cudaGraphDestroy(g); return rc; }
    if (e != cudaSuccess) return cuda_fail(s, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(s, e, "cudaGraphInstantiate");
    return PSS_OK;
}

void drop_graphs(pss_system *s) {
    for (cudaGraphExec_t &g : s->graphs)
        if (g) { cudaGraphExecDestroy(g); g = nullptr; }
    for (auto &pg : s->p2_graphs) cudaGraphExecDestroy(pg.second);
    s->p2_graphs.clear();
}

// The persistent path: runs of at most kMaxPersistSteps steps, one
// cooperative launch each.  The launch reads the product of the current state
// (array B, column-major, as the prologue or the previous launch left it) and
// leaves the state, the product of the new state and the next step's noise
// (XI) as the two-kernel path would, so the paths may alternate.
constexpr int64_t kMaxPersistSteps = 4096;

P2Args p2_args(pss_system *s, int nsteps) {
    P2Args a{};
    a.sp = sys_params<float>(s);
    a.fps = (const FieldP<float> *)s->fps;
    a.state = (float2 *)s->state;
    a.P = (float2 *)s->B;
    a.T1 = (float2 *)s->A;
    a.T1a = (float2 *)s->GS;
    a.xi = any_noisy(s) ? (float2 *)s->XI : nullptr;
    a.tw = (const float2 *)s->tw;
    a.d_step = s->d_step;
    a.d_status = s->d_status;
    a.gs = s->gs;
    a.nsteps = nsteps;
    a.prologue = (s->stale || !s->b_fast) ? 1 : 0;
    return a;
}

// The launch of a run of `len` steps, captured once into a graph of one
// kernel node and replayed (a graph launch costs the host less than a
// cooperative launch); the arguments depend only on len and the system's
// buffers and launch shape, so a graph stays valid until the system's
// launches change (invalidate).  If the capture is refused, every run
// launches directly.
constexpr size_t kMaxP2Graphs = 8;

cudaGraphExec_t p2_graph(pss_system *s, int len) {
    if (s->p2_capture <= 0) return nullptr;
    const P2Args args = p2_args(s, len);
    const int key = 2 * len + args.prologue;
    for (auto &pg : s->p2_graphs)
        if (pg.first == key) return pg.second;
    cudaError_t e = cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { cudaGetLastError(); s->p2_capture = -1; return nullptr; }
    cudaError_t el = launch_p2(args, s->nx, p2_radix(s), p2_blocks(s), p2_mode(s), s->cap_stream);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s->cap_stream, &g);
    cudaGraphExec_t ge = nullptr;
    if (el == cudaSuccess && e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
    if (g) cudaGraphDestroy(g);
    if (el != cudaSuccess || e != cudaSuccess || !ge) {
        cudaGetLastError();   // a refused capture leaves no error behind: launch directly from now on
        if (ge) cudaGraphExecDestroy(ge);
        s->p2_capture = -1;
        return nullptr;
    }
    if (s->p2_graphs.size() >= kMaxP2Graphs) {
        cudaGraphExecDestroy(s->p2_graphs.front().second);
        s->p2_graphs.erase(s->p2_graphs.begin());
    }
    s->p2_graphs.emplace_back(key, ge);
    return ge;
}

int run_persist(pss_system *s, int64_t n, cudaStream_t st) {
    if (!s->graph_valid) {
        drop_graphs(s);
        s->graph_valid = true;
    }
    for (int64_t done = 0; done < n;) {
        const int len = (int)std::min<int64_t>(kMaxPersistSteps, n - done);
        cudaGraphExec_t g = p2_graph(s, len);
        cudaError_t e = g ? cudaGraphLaunch(g, st)
                          : launch_p2(p2_args(s, len), s->nx, p2_radix(s), p2_blocks(s), p2_mode(s), st);
        s->launches++;
        if (e != cudaSuccess) return cuda_fail(s, e, "k2p_step launch");
        // the launch leaves the product of its last state in B (column-major) and the
        // next step's noise in XI, as the FP32 2D path keeps them
        s->stale = false;
        s->b_fast = true;
        done += len;
    }
    return PSS_OK;
}

// Every run of steps replays captured graphs: whole graphs of `graph_steps`
// steps, then one graph of the remaining length (captured on its first use
// and kept), so that the launches per step do not depend on n.
int run_steps(pss_system *s, int64_t n) {
    if (persist2d(s)) return run_persist(s, n, s->stream);
    const int chunk = s->tune_graph_steps > 0 ? s->tune_graph_steps : kDefaultGraphSteps;
    if (!s->graph_valid) {
        drop_graphs(s);
        s->graph_valid = true;
    }
    if ((int)s->graphs.size() < chunk + 1) s->graphs.resize(chunk + 1, nullptr);
    auto graph_of = [&](int len, cudaGraphExec_t *g) -> int {
        if (!s->graphs[len]) {
            int rc = capture_graph(&s, 1, len, &s->graphs[len]);
            if (rc) { s->graphs[len] = nullptr; return rc; }
        }
        *g = s->graphs[len];
        return PSS_OK;
    };
    int64_t done = 0;
    while (done < n) {
        const int len = (int)std::min<int64_t>(chunk, n - done);
        cudaGraphExec_t g = nullptr;
        if (int rc = graph_of(len, &g)) return rc;
        CK(cudaGraphLaunch(g, s->stream));
        s->launches += (int64_t)len * s->graph_launches;
        done += len;
    }
    return PSS_OK;
}

template <typename T> int timed_steps(pss_system *s, int64_t n, double *avg_ms) {
    Timer timer;
    Seq<T> q{s, s->cap_stream, 0, s->nslots(), &timer};
    CK(cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal));
    int rc = PSS_OK;
    for (int64_t k = 0; k < n && rc == PSS_OK; ++k) rc = q.one_step();
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(s->cap_stream, &g);
    if (rc) { if (g) cudaGraphDestroy(g); return rc; }
    if (e != cudaSuccess) return cuda_fail(s, e, "cudaStreamEndCapture");
    cudaGraphExec_t ge = nullptr;
    e = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(s, e, "cudaGraphInstantiate");
    e = cudaGraphLaunch(ge, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    cudaGraphExecDestroy(ge);
    if (e != cudaSuccess) return cuda_fail(s, e, "timed graph");
    for (int kind = 0; kind < 4; ++kind) {
        const auto &v = timer.ev[kind];
        double tot = 0;
        for (size_t i = 0; i + 1 < v.size(); i += 2) {
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, v[i], v[i + 1]));
            tot += ms;
        }
        avg_ms[kind] = v.size() >= 2 ? tot / (double)(v.size() / 2) : 0.0;
    }
    return PSS_OK;
}

int check_field(pss_system *s, int fid) {
    if (!s) return PSS_EINVAL;
    if (fid < 0 || fid >= (int)s->fields.size()) return fail(s, PSS_EINVAL, "no field %d", fid);
    return PSS_OK;
}

int cur_slot(const pss_system *s, int fid) { return s->cur * (int)s->fields.size() + fid; }

int ensure_real(pss_system *s) {
    if (!s->real) CK(cudaMalloc(&s->real, rsize(s) * (size_t)s->nsites));
    return PSS_OK;
}

int ensure_half(pss_system *s) {
    if (!s->half) CK(cudaMalloc(&s->half, csize(s) * (size_t)s->hx * s->ny * s->nz));
    return PSS_OK;
}

int device_errors(pss_system *s) {
    int st = 0;
    CK(cudaMemcpyAsync(&st, s->d_status, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    if (st) {
        CK(cudaMemsetAsync(s->d_status, 0, sizeof(int), s->stream));
        if (st & 2) {
            // a persistent launch that gave up leaves its barrier words behind
            CK(cudaMemsetAsync(s->gs, 0, sizeof(GridSync), s->stream));
            CK(cudaStreamSynchronize(s->stream));
            return fail(s, PSS_ETIMEOUT, "a bounded device wait ran out");
        }
        return fail(s, PSS_ENONFINITE, "a field became NaN or Inf");
    }
    return PSS_OK;
}

void invalidate(pss_system *s) {
    s->graph_valid = false;
    s->adj_graph_valid = false;
    s->gen++;
}


// (re)allocate the slot arrays for the current number of slots, keeping the
// data of the slots that exist
int grow_arrays(pss_system *s, int old_nf) {
    const int nf = (int)s->fields.size();
    const size_t slot_bytes = csize(s) * s->field_elems;
    void **arrays[3] = {&s->state, &s->A, &s->B};
    for (void **arr : arrays) {
        void *nb = nullptr;
        CK(cudaMalloc(&nb, slot_bytes * (size_t)s->batch * nf));
        CK(cudaMemset(nb, 0, slot_bytes * (size_t)s->batch * nf));
        if (*arr && old_nf > 0)
            for (int b = 0; b < s->batch; ++b)
                CK(cudaMemcpy((char *)nb + slot_bytes * ((size_t)b * nf), (char *)*arr + slot_bytes * ((size_t)b * old_nf),
                              slot_bytes * old_nf, cudaMemcpyDeviceToDevice));
        cudaFree(*arr);
        *arr = nb;
    }
    cudaFree(s->fps);
    s->fps = nullptr;
    cudaFree(s->XI);   // drawn-ahead noise of the fast 2D path: reallocated for the new slot count
    s->XI = nullptr;
    cudaFree(s->GS);
    s->GS = nullptr;
    CK(cudaMalloc(&s->fps, fpsize(s) * (size_t)s->batch * nf));
    s->fps_dirty = true;
    return PSS_OK;
}

int do_create(pss_system **out, int batch, int dim, int nx, int ny, int nz, double dx, double dy, double dz, double dt,
              const uint64_t *seeds, int precision) {
    if (!out) return fail(nullptr, PSS_EINVAL, "out is NULL");
    *out = nullptr;
    if (dim < 1 || dim > 3) return fail(nullptr, PSS_EINVAL, "dim must be 1, 2 or 3");
    if (batch < 1 || batch > kMaxBatch) return fail(nullptr, PSS_EINVAL, "batch must be in [1, %d]", kMaxBatch);
    if (!seeds) return fail(nullptr, PSS_EINVAL, "seeds is NULL");
    if (dim < 2) ny = 1;
    if (dim < 3) nz = 1;
    if (!pow2_in(nx, 4, 1024) || (dim >= 2 && !pow2_in(ny, 4, 1024)) || (dim == 3 && !pow2_in(nz, 4, 1024)))
        return fail(nullptr, PSS_EUNSUPPORTED, "sizes must be powers of two in [4, 1024]");
    if (!(dx > 0) || (dim >= 2 && !(dy > 0)) || (dim == 3 && !(dz > 0)) || !(dt > 0))
        return fail(nullptr, PSS_EINVAL, "spacings and dt must be positive");
    if (precision != PSS_F32 && precision != PSS_F64) return fail(nullptr, PSS_EINVAL, "precision");
    if ((long long)nx * ny * nz > (1ll << 30)) return fail(nullptr, PSS_EUNSUPPORTED, "lattice too large");
    pss_system *s = new pss_system();
    static std::atomic<uint64_t> next_uid{1};
    s->uid = next_uid++;
    s->dim = dim; s->nx = nx; s->ny = ny; s->nz = nz;
    s->dx[0] = dx; s->dx[1] = dim >= 2 ? dy : 1.0; s->dx[2] = dim == 3 ? dz : 1.0;
    s->dt = dt; s->prec = precision;
    s->batch = batch;
    s->seeds.assign(seeds, seeds + batch);
    s->hx = nx / 2 + 1;
    s->ntiles = (s->hx + kTileW - 1) / kTileW;
    s->rows = ny * nz;
    s->n_outer = dim == 3 ? ny : 1;
    s->n_inner = dim == 3 ? nz : (dim == 2 ? ny : 1);
    s->nsites = (long long)nx * ny * nz;
    s->field_elems = (size_t)s->ntiles * s->rows * kTileW;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_step, sizeof(long long));
    if (e == cudaSuccess) e = cudaMalloc(&s->d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(s->d_step, 0, sizeof(long long));
    if (e == cudaSuccess) e = cudaMemset(s->d_status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->coop, cudaDevAttrCooperativeLaunch, s->device);
    if (e == cudaSuccess) e = cudaMalloc(&s->gs, sizeof(GridSync));
    if (e == cudaSuccess) e = cudaMemset(s->gs, 0, sizeof(GridSync));
    // twiddle tables of every transform length and radix cap, built in FP64 on the host
    if (e == cudaSuccess) {
        const int total = kTwiddleEntries;
        std::vector<double2> h(total, make_double2(0.0, 0.0));
        for (int emax : {8, 16, 32})
            for (int n = 2; n <= kMaxFftN; n *= 2) {
                const int E = fft_E(n, emax);
                for (int P = E, R = std::min(E, n / P); P < n; P *= R, R = std::min(E, n / P))
                    for (int r = 1; r < R; ++r)
                        for (int k = 0; k < P; ++k) {
                            const double a = 2 * kPi * (double)(r * k) / (double)(P * R);
                            h[twiddle_offset(n, emax) + (P - E) + (r - 1) * P + k] = make_double2(std::cos(a), -std::sin(a));
                        }
            }
        if (precision == PSS_F64) {
            e = cudaMalloc(&s->tw, sizeof(double2) * total);
            if (e == cudaSuccess) e = cudaMemcpy(s->tw, h.data(), sizeof(double2) * total, cudaMemcpyHostToDevice);
        } else {
            std::vector<float2> hf(total);
            for (int m = 0; m < total; ++m) hf[m] = make_float2((float)h[m].x, (float)h[m].y);
            e = cudaMalloc(&s->tw, sizeof(float2) * total);
            if (e == cudaSuccess) e = cudaMemcpy(s->tw, hf.data(), sizeof(float2) * total, cudaMemcpyHostToDevice);
        }
    }
    if (e != cudaSuccess) {
        int rc = cuda_fail(nullptr, e, "pss_create_system");
        pss_destroy_system(s);
        return rc;
    }
    *out = s;
    return PSS_OK;
}

// per-slot real-space transfers go through the one-slot scratch
template <typename T> int forward_slot(pss_system *s, int slot) {
    return Seq<T>{s, s->stream, slot, 1}.forward_from_real();
}
template <typename T> int inverse_slot(pss_system *s, int slot) {
    return Seq<T>{s, s->stream, slot, 1}.inverse_to_real();
}

int forward_field(pss_system *s, int field_id) {
    int rc = upload_params(s);
    if (rc) return rc;
    const int slot = cur_slot(s, field_id);
    rc = s->prec == PSS_F64 ? forward_slot<double>(s, slot) : forward_slot<float>(s, slot);
    s->stale = true;
    return rc;
}

int adj_alloc(pss_system *s, int64_t nck, int64_t K) {
    const size_t slot_bytes = csize(s) * s->field_elems;
    cudaFree(s->ck);
    cudaFree(s->seg);
    cudaFree(s->seg_prod);
    cudaFree(s->seg_real);
    cudaFree(s->seg_noise);
    s->ck = s->seg = s->seg_prod = s->seg_real = s->seg_noise = nullptr;
    CK(cudaMalloc(&s->ck, slot_bytes * (size_t)(nck + 1)));
    CK(cudaMalloc(&s->seg, slot_bytes * (size_t)(K + 1)));
    CK(cudaMalloc(&s->seg_prod, slot_bytes * (size_t)(K + 1)));
    CK(cudaMalloc(&s->seg_real, rsize(s) * (size_t)s->nsites * (size_t)(K + 1)));
    if (persist2d_ok(s)) CK(cudaMalloc(&s->seg_noise, slot_bytes * (size_t)(K + 1)));
    if (!s->L) CK(cudaMalloc(&s->L, slot_bytes));
    if (!s->d_grad) CK(cudaMalloc(&s->d_grad, sizeof(double) * 11));
    if (!s->d_seg) CK(cudaMalloc(&s->d_seg, sizeof(long long) * 2));
    if (s->adj_graph) cudaGraphExecDestroy(s->adj_graph);
    s->adj_graph = nullptr;
    s->adj_graph_valid = false;
    return PSS_OK;
}

int copy_slot(pss_system *s, void *dst, const void *src) {
    CK(cudaMemcpyAsync(dst, src, csize(s) * s->field_elems, cudaMemcpyDeviceToDevice, s->stream));
    return PSS_OK;
}

void *slot_ptr(const pss_system *s, void *base, int64_t i) { return (char *)base + csize(s) * s->field_elems * i; }

// One segment of the backward pass, of len steps: recompute it from checkpoint
// *d_seg, keeping every state, its product and its real field, then run its
// adjoint steps, last first.  The segment index is read on the device, so one
// captured graph serves every full segment.
template <typename T> int record_adjoint_segment(pss_system *s, cudaStream_t stream, int64_t len) {
    Seq<T> q{s, stream, 0, 1};
    auto st = [&](int64_t i) { return (cplx<T> *)slot_ptr(s, s->seg, i); };
    auto prod = [&](int64_t i) { return (cplx<T> *)slot_ptr(s, s->seg_prod, i); };
    auto real = [&](int64_t i) { return (T *)s->seg_real + (size_t)s->nsites * (size_t)i; };
    cudaError_t e = launch_segment_begin<T>(st(0), (const cplx<T> *)s->ck, s->field_elems, s->d_seg,
                                            (long long)s->adj_step0, (long long)s->adj_K, s->d_step, s->d_seg + 1,
                                            stream);
    s->launches++;
    if (e != cudaSuccess) return cuda_fail(s, e, "segment start kernel");
    int rc;
    if (persist2d(s) && len >= 1) {
        // the segment's forward steps as one persistent launch that writes every
        // step's state, product and de-aliased real field (segment mode)
        P2Args a = p2_args(s, (int)len);
        a.state = (float2 *)st(0);
        a.P = nullptr;
        a.xi = nullptr;
        a.prologue = 1;
        a.seg_state = (float2 *)st(0);
        a.seg_prod = (float2 *)prod(0);
        a.seg_real = (float *)real(0);
        a.seg_noise = s->tune_persist_adj ? (float2 *)s->seg_noise : nullptr;
        a.seg_cstride = s->field_elems;
        a.seg_rstride = (size_t)s->nsites;
        e = launch_p2(a, s->nx, p2_radix(s), p2_blocks(s), 0, stream);
        s->launches++;
        if (e != cudaSuccess) return cuda_fail(s, e, "k2p_step launch (recomputed segment)");
        if (s->tune_persist_adj && s->seg_noise) {
            // the segment's backward pass as one persistent launch (k2p_adj): the adjoint
            // field from L and back, nu and w through A and B
            P2AdjArgs b{};
            b.sp = a.sp;
            b.fps = a.fps;
            b.tw = a.tw;
            b.L = (float2 *)s->L;
            b.NU = (float2 *)s->A;
            b.W = (float2 *)s->B;
            b.seg_state = (const float2 *)st(0);
            b.seg_prod = (const float2 *)prod(0);
            b.seg_real = (const float *)real(0);
            b.seg_noise = (const float2 *)s->seg_noise;
            b.cstride = s->field_elems;
            b.rstride = (size_t)s->nsites;
            b.grad = s->d_grad;
            b.d_status = s->d_status;
            b.gs = s->gs;
            b.len = (int)len;
            e = launch_p2_adj(b, s->nx, s->tune_adj_radix ? s->tune_adj_radix : p2_radix(s), p2_blocks(s), stream);
            s->launches++;
            if (e != cudaSuccess) return cuda_fail(s, e, "k2p_adj launch");
            return PSS_OK;
        }
    } else {
        if ((rc = q.recompute_prologue(st(0), prod(0), real(0)))) return rc;
        for (int64_t i = 0; i < len; ++i)
            if ((rc = q.recompute_step(st(i), st(i + 1), prod(i), prod(i + 1), real(i + 1)))) return rc;
    }
    if (len < 1 || !q.fused_adjoint()) {
        for (int64_t i = len - 1; i >= 0; --i)
            if ((rc = q.adjoint_step(st(i + 1), prod(i), real(i), i))) return rc;
        return PSS_OK;
    }
    if ((rc = q.adjoint_part_a(st(len), prod(len - 1), len - 1))) return rc;
    for (int64_t i = len - 1; i >= 1; --i) {
        if ((rc = q.adjoint_x_part(real(i)))) return rc;
        if ((rc = q.adjoint_part_ba(st(i), prod(i - 1), i))) return rc;
    }
    if ((rc = q.adjoint_x_part(real(0)))) return rc;
    return q.adjoint_part_b(0);
}

template <typename T> int adjoint_backward_t(pss_system *s) {
    for (int64_t j = s->adj_nck - 1; j >= 0; --j) {
        const int64_t len = std::min<int64_t>(s->adj_K, s->adj_n - j * s->adj_K);
        cudaError_t e = launch_set_i64(s->d_seg, (long long)j, s->stream);
        s->launches++;
        if (e != cudaSuccess) return cuda_fail(s, e, "segment index kernel");
        int rc;
        if (len == s->adj_K && s->adj_nck > 1) {
            if (!s->adj_graph_valid) {
                if (s->adj_graph) { cudaGraphExecDestroy(s->adj_graph); s->adj_graph = nullptr; }
                CK(cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal));
                const int64_t before = s->launches;
                rc = record_adjoint_segment<T>(s, s->cap_stream, len);
                s->adj_graph_launches = s->launches - before;
                s->launches = before;
                cudaGraph_t g = nullptr;
                e = cudaStreamEndCapture(s->cap_stream, &g);
                if (rc) { if (g) cudaGraphDestroy(g); return rc; }
                if (e != cudaSuccess) return cuda_fail(s, e, "cudaStreamEndCapture");
                e = cudaGraphInstantiate(&s->adj_graph, g, 0);
                cudaGraphDestroy(g);
                if (e != cudaSuccess) return cuda_fail(s, e, "cudaGraphInstantiate");
                s->adj_graph_valid = true;
            }
            CK(cudaGraphLaunch(s->adj_graph, s->stream));
            s->launches += s->adj_graph_launches;
        } else if ((rc = record_adjoint_segment<T>(s, s->stream, len))) {
            return rc;
        }
    }
    return PSS_OK;
}

}  // namespace

// ==========================================================================
// C ABI
// ==========================================================================
extern "C" {

int pss_create_system(pss_system **out, int dim, int nx, int ny, int nz, double dx, double dy, double dz,
                      double dt, uint64_t seed, int precision) {
    return do_create(out, 1, dim, nx, ny, nz, dx, dy, dz, dt, &seed, precision);
}

int pss_create_batch(pss_system **out, int batch, int dim, int nx, int ny, int nz, double dx, double dy, double dz,
                     double dt, const uint64_t *seeds, int precision) {
    return do_create(out, batch, dim, nx, ny, nz, dx, dy, dz, dt, seeds, precision);
}

int pss_destroy_system(pss_system *s) {
    if (!s) return PSS_OK;
    drop_graphs(s);
    for (auto &m : s->many) if (m.exec) cudaGraphExecDestroy(m.exec);
    cudaFree(s->state);
    cudaFree(s->A);
    cudaFree(s->B);
    cudaFree(s->XI);
    cudaFree(s->GS);
    cudaFree(s->real_acc);
    cudaFree(s->real_tp);
    cudaFree(s->fps);
    cudaFree(s->tw);
    cudaFree(s->real);
    cudaFree(s->half);
    cudaFree(s->sq);
    cudaFree(s->d_step);
    cudaFree(s->d_status);
    cudaFree(s->gs);
    cudaFree(s->L);
    cudaFree(s->ck);
    cudaFree(s->seg);
    cudaFree(s->seg_prod);
    cudaFree(s->seg_real);
    cudaFree(s->seg_noise);
    cudaFree(s->d_grad);
    cudaFree(s->d_seg);
    if (s->adj_graph) cudaGraphExecDestroy(s->adj_graph);
    if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
    delete s;
    return PSS_OK;
}

int pss_set_stream(pss_system *s, void *stream) {
    if (!s) return PSS_EINVAL;
    cudaStream_t next = (cudaStream_t)stream;
    if (next != s->stream) {
        // work issued on the new stream starts after everything issued so far
        cudaEvent_t ev;
        CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        cudaError_t e = cudaEventRecord(ev, s->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(next, ev, 0);
        cudaEventDestroy(ev);
        if (e != cudaSuccess) return cuda_fail(s, e, "pss_set_stream");
        s->stream = next;
    }
    return PSS_OK;
}

int pss_add_param(pss_system *s, const char *name, double value, int *id) {
    if (!s || !name) return s ? fail(s, PSS_EINVAL, "name is NULL") : PSS_EINVAL;
    for (const std::string &p : s->param_names)
        if (p == name) return fail(s, PSS_EINVAL, "parameter '%s' exists", name);
    const size_t np = s->param_names.size();
    std::vector<double> v((np + 1) * s->batch);
    for (int b = 0; b < s->batch; ++b) {
        for (size_t i = 0; i < np; ++i) v[b * (np + 1) + i] = s->param_values[b * np + i];
        v[b * (np + 1) + np] = value;
    }
    s->param_values.swap(v);
    s->param_names.push_back(name);
    if (id) *id = (int)np;
    s->fps_dirty = true;
    return PSS_OK;
}

int pss_set_param(pss_system *s, int id, double value) {
    if (!s) return PSS_EINVAL;
    if (id < 0 || id >= (int)s->param_names.size()) return fail(s, PSS_EINVAL, "no parameter %d", id);
    for (int b = 0; b < s->batch; ++b) s->param_values[(size_t)b * s->param_names.size() + id] = value;
    s->fps_dirty = true;
    if (!s->gterms.empty()) {
        // product-term operators are launch arguments, and a field with several
        // of them holds its next product with the operators applied
        invalidate(s);
        s->stale = true;
    }
    return PSS_OK;
}

int pss_set_param_batch(pss_system *s, int id, const double *values) {
    if (!s || !values) return PSS_EINVAL;
    if (id < 0 || id >= (int)s->param_names.size()) return fail(s, PSS_EINVAL, "no parameter %d", id);
    for (int b = 0; b < s->batch; ++b) s->param_values[(size_t)b * s->param_names.size() + id] = values[b];
    s->fps_dirty = true;
    if (!s->gterms.empty()) {
        invalidate(s);
        s->stale = true;
    }
    return PSS_OK;
}

int pss_get_param(pss_system *s, int id, double *value) {
    if (!s || !value) return PSS_EINVAL;
    if (id < 0 || id >= (int)s->param_names.size()) return fail(s, PSS_EINVAL, "no parameter %d", id);
    *value = pval(s, s->cur, id);
    return PSS_OK;
}

int pss_select_instance(pss_system *s, int instance) {
    if (!s) return PSS_EINVAL;
    if (instance < 0 || instance >= s->batch) return fail(s, PSS_EINVAL, "no instance %d", instance);
    s->cur = instance;
    return PSS_OK;
}

int pss_batch_size(const pss_system *s) { return s ? s->batch : 0; }

int pss_add_field(pss_system *s, const char *name, int dynamic, int *field_id) {
    if (!s || !name) return s ? fail(s, PSS_EINVAL, "name is NULL") : PSS_EINVAL;
    if (!dynamic) return fail(s, PSS_EUNSUPPORTED, "only dynamic fields are implemented");
    if ((int)s->fields.size() >= kMaxFields) return fail(s, PSS_EUNSUPPORTED, "at most %d fields", kMaxFields);
    for (const Field &f : s->fields)
        if (f.name == name) return fail(s, PSS_EINVAL, "field '%s' exists", name);
    const int old_nf = (int)s->fields.size();
    Field f;
    f.name = name;
    s->fields.push_back(f);
    int rc = grow_arrays(s, old_nf);
    if (rc) {
        s->fields.pop_back();
        return rc;
    }
    if (field_id) *field_id = old_nf;
    s->stale = true;
    invalidate(s);
    return PSS_OK;
}

int pss_add_term(pss_system *s, int field_id, int implicit, int n_mono, const int *param_ids, const double *scales,
                 const int *q2_pows, int n_factors, const int *factor_fields, const int *powers) {
    int rc = check_field(s, field_id);
    if (rc) return rc;
    if (n_mono < 1 || n_mono > 8 || !scales || !q2_pows) return fail(s, PSS_EINVAL, "need 1..8 monomials");
    for (int m = 0; m < n_mono; ++m) {
        if (q2_pows[m] < 0 || q2_pows[m] >= kPolyTerms) return fail(s, PSS_EINVAL, "q^2 power must be in [0, 4]");
        const int pid = param_ids ? param_ids[m] : -1;
        if (pid >= (int)s->param_names.size()) return fail(s, PSS_EINVAL, "no parameter %d", pid);
    }
    if (n_factors < 1 || !factor_fields || !powers) return fail(s, PSS_EINVAL, "need at least one factor");
    if (n_factors != 1 || factor_fields[0] != field_id)
        return fail(s, PSS_EUNSUPPORTED, "terms must be a power of the field itself in this build");
    const int p = powers[0];
    Field &f = s->fields[field_id];
    if (implicit) {
        if (p != 1) return fail(s, PSS_EINVAL, "implicit terms must be linear in the field");
        for (int m = 0; m < n_mono; ++m) f.lhs.push_back({param_ids ? param_ids[m] : -1, scales[m], q2_pows[m]});
    } else {
        if (p < 1 || p > 3) return fail(s, PSS_EUNSUPPORTED, "explicit products must be a power 1..3");
        if (f.power != 0 && f.power != p) return fail(s, PSS_EUNSUPPORTED, "explicit terms of a field share one power");
        f.power = p;
        for (int m = 0; m < n_mono; ++m) f.rhs.push_back({param_ids ? param_ids[m] : -1, scales[m], q2_pows[m]});
    }
    s->stale = true;
    s->fps_dirty = true;
    return PSS_OK;
}

int check_monos(pss_system *s, int n_mono, const int *param_ids, const double *scales, const int *q2_pows) {
    if (n_mono < 1 || n_mono > 8 || !scales || !q2_pows) return fail(s, PSS_EINVAL, "need 1..8 monomials");
    for (int m = 0; m < n_mono; ++m) {
        if (q2_pows[m] < 0 || q2_pows[m] >= kPolyTerms) return fail(s, PSS_EINVAL, "q^2 power must be in [0, 4]");
        const int pid = param_ids ? param_ids[m] : -1;
        if (pid >= (int)s->param_names.size()) return fail(s, PSS_EINVAL, "no parameter %d", pid);
    }
    return PSS_OK;
}

int add_gterm(pss_system *s, GTerm t) {
    s->gterms.push_back(std::move(t));
    s->fields[s->gterms.back().target].general = true;
    s->stale = true;
    s->fps_dirty = true;
    invalidate(s);
    return PSS_OK;
}

int pss_add_product_term(pss_system *s, int field_id, int n_mono, const int *param_ids, const double *scales,
                         const int *q2_pows, int n_factors, const int *factor_fields, const int *powers,
                         const int *derivs, const int *laps) {
    int rc = check_field(s, field_id);
    if (rc) return rc;
    if ((rc = check_monos(s, n_mono, param_ids, scales, q2_pows))) return rc;
    if (n_factors < 1 || n_factors > 8 || !factor_fields || !powers)
        return fail(s, PSS_EINVAL, "need 1..8 factors");
    GTerm t{field_id, {}, {}};
    for (int m = 0; m < n_mono; ++m) t.M.push_back({param_ids ? param_ids[m] : -1, scales[m], q2_pows[m]});
    for (int k = 0; k < n_factors; ++k) {
        const int fld = factor_fields[k], pw = powers[k], d = derivs ? derivs[k] : -1, l = laps ? laps[k] : 0;
        if (fld < 0 || fld >= (int)s->fields.size()) return fail(s, PSS_EINVAL, "no field %d", fld);
        if (pw < 1 || pw > 4) return fail(s, PSS_EINVAL, "factor powers are 1..4");
        if (d < -1 || d >= s->dim) return fail(s, PSS_EINVAL, "derivative axis must be -1 or 0..dim-1");
        if (l < 0 || l > 2) return fail(s, PSS_EINVAL, "Laplacian powers are 0..2");
        t.factors.push_back({fld, pw, d, l});
    }
    return add_gterm(s, std::move(t));
}

int pss_add_grad_sq_term(pss_system *s, int field_id, int n_mono, const int *param_ids, const double *scales,
                         const int *q2_pows) {
    int rc = check_field(s, field_id);
    if (rc) return rc;
    if ((rc = check_monos(s, n_mono, param_ids, scales, q2_pows))) return rc;
    // sum_j (d_j phi)^2: one term per axis, all with the same operator
    for (int j = 0; j < s->dim; ++j) {
        GTerm t{field_id, {}, {{field_id, 2, j, 0}}};
        for (int m = 0; m < n_mono; ++m) t.M.push_back({param_ids ? param_ids[m] : -1, scales[m], q2_pows[m]});
        add_gterm(s, std::move(t));
    }
    return PSS_OK;
}

int pss_set_noise(pss_system *s, int field_id, int D_param_id, int q2_pow) {
    int rc = check_field(s, field_id);
    if (rc) return rc;
    if (D_param_id < 0 || D_param_id >= (int)s->param_names.size())
        return fail(s, PSS_EINVAL, "no parameter %d", D_param_id);
    if (q2_pow < 0 || q2_pow >= kPolyTerms) return fail(s, PSS_EINVAL, "q^2 power must be in [0, 4]");
    Field &f = s->fields[field_id];
    f.noisy = true;
    f.noise_param = D_param_id;
    f.noise_pow = q2_pow;
    s->fps_dirty = true;
    s->stale = true;   // the fast 2D path keeps the next step's noise drawn ahead
    invalidate(s);
    return PSS_OK;
}

int pss_set_dealias(pss_system *s, int field_id, int order) {
    int rc = check_field(s, field_id);
    if (rc) return rc;
    if (order < 0) return fail(s, PSS_EINVAL, "order must be >= 0");
    s->fields[field_id].dealias = order;
    s->stale = true;
    s->fps_dirty = true;
    invalidate(s);   // the number of kept tiles is baked into the launches
    return PSS_OK;
}

int pss_set_frame(pss_system *s, int field_id, int width, double lo_value, double hi_value) {
    int rc = check_field(s, field_id);
    if (rc) return rc;
    if (width < 0 || 2 * width > s->nx) return fail(s, PSS_EINVAL, "frame width must be in [0, Nx/2]");
    if (!std::isfinite(lo_value) || !std::isfinite(hi_value)) return fail(s, PSS_EINVAL, "frame values must be finite");
    Field &f = s->fields[field_id];
    f.frame_w = width;
    f.frame_lo = lo_value;
    f.frame_hi = hi_value;
    invalidate(s);
    return PSS_OK;
}

int pss_set_field(pss_system *s, int field_id, const void *real, int where) {
    int rc = check_field(s, field_id);
    if (rc) return rc;
    if (!real) return fail(s, PSS_EINVAL, "real is NULL");
    if ((rc = ensure_real(s))) return rc;
    const size_t bytes = rsize(s) * (size_t)s->nsites;
    CK(cudaMemcpyAsync(s->real, real, bytes, where == PSS_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                       s->stream));
    return forward_field(s, field_id);
}

int pss_init_uniform(pss_system *s, int field_id, double lo, double hi) {
    int rc = check_field(s, field_id);
    if (rc) return rc;
    if ((rc = ensure_real(s))) return rc;
    const uint64_t seed = s->seeds[s->cur];
    cudaError_t e = s->prec == PSS_F64
        ? launch_init_uniform<double>((double *)s->real, s->nsites, lo, hi, seed, field_id, s->stream)
        : launch_init_uniform<float>((float *)s->real, s->nsites, lo, hi, seed, field_id, s->stream);
    s->launches++;
    if (e != cudaSuccess) return cuda_fail(s, e, "init kernel");
    return forward_field(s, field_id);
}

int pss_step(pss_system *s, int64_t n) {
    if (!s) return PSS_EINVAL;
    if (n < 0) return fail(s, PSS_EINVAL, "n must be >= 0");
    if (s->fields.empty()) return fail(s, PSS_EINVAL, "no fields");
    if (n == 0) return PSS_OK;
    int rc = upload_params(s);
    if (rc) return rc;
    if (round_trip(s) && (rc = ensure_real(s))) return rc;
    if ((rc = prologue(s, persist2d(s)))) return rc;
    if ((rc = run_steps(s, n))) return rc;
    s->step += n;
    return PSS_OK;
}

int pss_step_many(pss_system **systems, int n, int64_t steps) {
    if (!systems || n < 1) return fail(nullptr, PSS_EINVAL, "need at least one system");
    pss_system *s0 = systems[0];
    if (!s0) return fail(nullptr, PSS_EINVAL, "systems[0] is NULL");
    if (steps < 0) return fail(s0, PSS_EINVAL, "steps must be >= 0");
    for (int i = 0; i < n; ++i) {
        pss_system *s = systems[i];
        if (!s || s->fields.empty()) return fail(s0, PSS_EINVAL, "system %d has no fields", i);
        if (i > 0) {
            int rc = pss_set_stream(s, s0->stream);
            if (rc) return fail(s0, rc, "%s", s->err.c_str());
        }
        int rc = upload_params(s);
        if (!rc && round_trip(s)) rc = ensure_real(s);
        if (!rc) rc = prologue(s);
        if (rc) return i == 0 ? rc : fail(s0, rc, "%s", s->err.c_str());
    }
    if (steps == 0) return PSS_OK;
    const int chunk = s0->tune_graph_steps > 0 ? s0->tune_graph_steps : kDefaultGraphSteps;
    // graphs of whole chunks and of the remainder, kept on systems[0] for this
    // list of systems as long as none of them changed its launches
    auto graph_of = [&](int len, cudaGraphExec_t *out) -> int {
        std::vector<uint64_t> uids(n), gens(n);
        for (int i = 0; i < n; ++i) { uids[i] = systems[i]->uid; gens[i] = systems[i]->gen; }
        for (auto &m : s0->many)
            if (m.len == len && m.uids == uids && m.gens == gens) {
                m.stamp = ++s0->many_clock;
                *out = m.exec;
                return PSS_OK;
            }
        cudaGraphExec_t ge = nullptr;
        int rc = capture_graph(systems, n, len, &ge);
        if (rc) return rc;
        constexpr size_t kKeep = 8;
        if (s0->many.size() >= kKeep) {   // the least recently used entry goes
            size_t old = 0;
            for (size_t k = 1; k < s0->many.size(); ++k)
                if (s0->many[k].stamp < s0->many[old].stamp) old = k;
            cudaGraphExecDestroy(s0->many[old].exec);
            s0->many.erase(s0->many.begin() + (long)old);
        }
        pss_system::Many m;
        m.uids = uids;
        m.gens = gens;
        m.len = len;
        m.exec = ge;
        m.stamp = ++s0->many_clock;
        s0->many.push_back(m);
        *out = ge;
        return PSS_OK;
    };
    int64_t done = 0;
    while (done < steps) {
        const int len = (int)std::min<int64_t>(chunk, steps - done);
        cudaGraphExec_t ge = nullptr;
        if (int rc = graph_of(len, &ge)) return rc;
        cudaError_t e = cudaGraphLaunch(ge, s0->stream);
        if (e != cudaSuccess) return cuda_fail(s0, e, "cudaGraphLaunch");
        for (int i = 0; i < n; ++i) systems[i]->launches += (int64_t)len * systems[i]->graph_launches;
        done += len;
    }
    for (int i = 0; i < n; ++i) systems[i]->step += steps;
    return PSS_OK;
}

int pss_adjoint_forward(pss_system *s, int64_t n) {
    if (!s) return PSS_EINVAL;
    if (n < 1) return fail(s, PSS_EINVAL, "n must be >= 1");
    if (s->nslots() != 1) return fail(s, PSS_EUNSUPPORTED, "the adjoint needs one field and batch 1 in this build");
    if (round_trip(s)) return fail(s, PSS_EUNSUPPORTED, "the adjoint has no boundary frames or real-space round trip");
    if (any_general(s)) return fail(s, PSS_EUNSUPPORTED, "the adjoint covers power products only");
    int64_t K = (int64_t)std::ceil(std::sqrt((double)n));
    const int64_t nck = (n + K - 1) / K;
    int rc = adj_alloc(s, nck, K);
    if (rc) return rc;
    s->adj_ready = false;
    s->adj_n = n;
    s->adj_step0 = s->step;
    s->adj_K = K;
    s->adj_nck = nck;
    for (int64_t j = 0; j < nck; ++j) {
        if ((rc = copy_slot(s, slot_ptr(s, s->ck, j), s->state))) return rc;
        if ((rc = pss_step(s, std::min<int64_t>(K, n - j * K)))) return rc;
    }
    if ((rc = copy_slot(s, slot_ptr(s, s->ck, nck), s->state))) return rc;
    s->adj_ready = true;
    return PSS_OK;
}

int pss_adjoint_backward(pss_system *s, const void *lambda_T, int where, double *dJ_dparams, void *lambda_0,
                         int where0) {
    if (!s || !lambda_T) return PSS_EINVAL;
    if (!s->adj_ready) return fail(s, PSS_EINVAL, "call pss_adjoint_forward first");
    int rc = upload_params(s);
    if (rc) return rc;
    // lambda_T (half spectrum) -> L (tiles)
    if ((rc = ensure_half(s))) return rc;
    const size_t hbytes = csize(s) * (size_t)s->hx * s->ny * s->nz;
    CK(cudaMemcpyAsync(s->half, lambda_T, hbytes, where == PSS_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                       s->stream));
    CK(cudaMemsetAsync(s->L, 0, csize(s) * s->field_elems, s->stream));
    cudaError_t e = s->prec == PSS_F64
        ? launch_half_to_tiles<double>(sys_params<double>(s), (const double2 *)s->half, (double2 *)s->L, s->stream)
        : launch_half_to_tiles<float>(sys_params<float>(s), (const float2 *)s->half, (float2 *)s->L, s->stream);
    s->launches++;
    if (e != cudaSuccess) return cuda_fail(s, e, "layout kernel");
    CK(cudaMemsetAsync(s->d_grad, 0, sizeof(double) * 11, s->stream));
    rc = s->prec == PSS_F64 ? adjoint_backward_t<double>(s) : adjoint_backward_t<float>(s);
    if (rc) return rc;
    // gradients of the named parameters
    double g[11];
    CK(cudaMemcpyAsync(g, s->d_grad, sizeof g, cudaMemcpyDeviceToHost, s->stream));
    if (lambda_0) {
        e = s->prec == PSS_F64
            ? launch_tiles_to_half<double>(sys_params<double>(s), (const double2 *)s->L, (double2 *)s->half, s->stream)
            : launch_tiles_to_half<float>(sys_params<float>(s), (const float2 *)s->L, (float2 *)s->half, s->stream);
        s->launches++;
        if (e != cudaSuccess) return cuda_fail(s, e, "layout kernel");
        CK(cudaMemcpyAsync(lambda_0, s->half, hbytes, where0 == PSS_HOST ? cudaMemcpyDeviceToHost
                                                                          : cudaMemcpyDeviceToDevice, s->stream));
    }
    // back to the state after the forward run
    if ((rc = copy_slot(s, s->state, slot_ptr(s, s->ck, s->adj_nck)))) return rc;
    long long st = s->adj_step0 + s->adj_n;
    CK(cudaMemcpyAsync(s->d_step, &st, sizeof st, cudaMemcpyHostToDevice, s->stream));
    s->step = st;
    s->stale = true;
    if ((rc = device_errors(s))) return rc;
    if (dJ_dparams) {
        const Field &f = s->fields[0];
        for (size_t i = 0; i < s->param_names.size(); ++i) dJ_dparams[i] = 0.0;
        for (const Mono &m : f.lhs)
            if (m.param >= 0) dJ_dparams[m.param] += m.scale * g[m.pow];
        for (const Mono &m : f.rhs)
            if (m.param >= 0) dJ_dparams[m.param] += m.scale * g[5 + m.pow];
        if (f.noisy && f.noise_param >= 0) {
            const double D = pval(s, 0, f.noise_param);
            if (D > 0) dJ_dparams[f.noise_param] += g[10] / (2.0 * D);
        }
    }
    return PSS_OK;
}

int pss_time_kernels(pss_system *s, int64_t n, double *avg_ms) {
    if (!s || !avg_ms) return PSS_EINVAL;
    if (n < 1) return fail(s, PSS_EINVAL, "n must be >= 1");
    if (s->fields.empty()) return fail(s, PSS_EINVAL, "no fields");
    int rc = upload_params(s);
    if (rc) return rc;
    if ((rc = prologue(s, persist2d(s)))) return rc;
    if (persist2d(s)) {
        // one launch of n steps between two events: its duration per step
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        CK(cudaEventCreate(&e0));
        cudaError_t e = cudaEventCreate(&e1);
        if (e == cudaSuccess) e = cudaEventRecord(e0, s->stream);
        if (e == cudaSuccess) {
            const int len = (int)std::min<int64_t>(n, kMaxPersistSteps);
            e = launch_p2(p2_args(s, len), s->nx, p2_radix(s), p2_blocks(s), p2_mode(s), s->stream);
            s->launches++;
            if (e == cudaSuccess) { s->stale = false; s->b_fast = true; }
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, s->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (e != cudaSuccess) return cuda_fail(s, e, "timed persistent launch");
        n = std::min<int64_t>(n, kMaxPersistSteps);
        avg_ms[0] = ms / (double)n;
        avg_ms[1] = avg_ms[2] = avg_ms[3] = 0.0;
    } else {
        rc = s->prec == PSS_F64 ? timed_steps<double>(s, n, avg_ms) : timed_steps<float>(s, n, avg_ms);
        if (rc) return rc;
    }
    s->step += n;
    return device_errors(s);
}

int pss_set_tuning(pss_system *s, const char *key, int value) {
    if (!s || !key) return PSS_EINVAL;
    if (value < 0) return fail(s, PSS_EINVAL, "tuning values are >= 0");
    const std::string k = key;
    if (k == "pdl") s->tune_pdl = value ? 1 : 0;
    else if (k == "row_pairs") s->tune_row_pairs = value;
    else if (k == "col_tiles") s->tune_col_tiles = value;
    else if (k == "mid_planes") s->tune_mid_planes = value;
    else if (k == "graph_steps") s->tune_graph_steps = value;
    else if (k == "fast2d") s->tune_fast2d = value ? 1 : 0;
    else if (k == "fast3d") s->tune_fast3d = value ? 1 : 0;
    else if (k == "fuse_adjoint") s->tune_fuse_adj = value ? 1 : 0;
    else if (k == "real_state") s->tune_real_state = value ? 1 : 0;
    else if (k == "test_timeout") s->tune_test_timeout = value ? 1 : 0;
    else if (k == "persist") s->tune_persist = value ? 1 : 0;
    else if (k == "adj_col2") s->tune_adj_col2 = value ? 1 : 0;
    else if (k == "persist_adj") s->tune_persist_adj = value ? 1 : 0;
    else if (k == "adj_radix") {
        if (value != 0 && value != 8 && value != 16) return fail(s, PSS_EINVAL, "adj_radix is 8 or 16 (0 = automatic)");
        s->tune_adj_radix = value;
    }
    else if (k == "persist_blocks") {
        if (value > 1024) return fail(s, PSS_EINVAL, "persist_blocks is at most 1024 (0 = automatic)");
        s->tune_persist_blocks = value;
    }
    else if (k == "col2_warps") {
        if (value > 24) return fail(s, PSS_EINVAL, "col2_warps is at most 24 (0 = automatic)");
        s->tune_col2_warps = value;
    }
    else if (k == "row2_pairs") s->tune_row2_pairs = value;
    else if (k == "adj_row_pairs") s->tune_adj_row_pairs = value;
    else if (k == "row2_share") {
        if (value > 100) return fail(s, PSS_EINVAL, "row2_share is a percentage");
        s->tune_row2_share = value;
    }
    else if (k == "row2_noise") {
        if (value > 24) return fail(s, PSS_EINVAL, "row2_noise is at most 24 (0 = automatic)");
        s->tune_row2_noise = value;
    }
    else if (k == "col2_radix" || k == "row2_radix") {
        if (value != 0 && value != 8 && value != 16 && value != 32)
            return fail(s, PSS_EINVAL, "radix 8, 16 or 32 (0 = automatic; 32 for sides of 1024 only)");
        (k == "col2_radix" ? s->tune_col2_radix : s->tune_row2_radix) = value;
    }
    else if (k == "col_radix" || k == "row_radix" || k == "mid_radix") {
        if (value != 0 && value != 8 && value != 16) return fail(s, PSS_EINVAL, "radix caps are 8 or 16 (0 = automatic)");
        (k == "col_radix" ? s->tune_col_radix : k == "row_radix" ? s->tune_row_radix : s->tune_mid_radix) = value;
    }
    else return fail(s, PSS_EINVAL, "unknown tuning key '%s'", key);
    invalidate(s);
    return PSS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Launch-shape autotuner.  Coordinate descent over the knobs of the system's
// step path: each knob in turn takes every value of its list with the others
// held at their best so far, and keeps the value whose timed run of steps is
// fastest (by more than 1 %, so that timing noise does not move it).  The
// lists hold only values the launch-shape tests run (the helpers above clamp
// them to the kernels' thread limits).
// ---------------------------------------------------------------------------
namespace {

struct TuneKnob {
    const char *name;
    int pss_system::*field;
    std::vector<int> values;
};

std::vector<TuneKnob> tune_space(const pss_system *s) {
    std::vector<TuneKnob> k;
    const auto radix_list = [](int side) { return side == 1024 ? std::vector<int>{8, 16, 32} : std::vector<int>{8, 16}; };
    if (fast2d(s)) {
        // the persistent launch against the two-kernel step, where the system qualifies
        if (persist2d_ok(s)) k.push_back({"persist", &pss_system::tune_persist, {1, 0}});
        k.push_back({"col2_radix", &pss_system::tune_col2_radix, radix_list(s->ny)});
        k.push_back({"row2_radix", &pss_system::tune_row2_radix, radix_list(s->nx)});
        k.push_back({"row2_pairs", &pss_system::tune_row2_pairs, {1, 2, 4, 8}});
        k.push_back({"col2_warps", &pss_system::tune_col2_warps, {4, 8, 16}});
        if (any_noisy(s)) k.push_back({"row2_noise", &pss_system::tune_row2_noise, {8, 16}});
    } else {
        k.push_back({"col_radix", &pss_system::tune_col_radix, {8, 16}});
        if (fast3d_rows(s)) k.push_back({"row2_radix", &pss_system::tune_row2_radix, {8, 16}});
        else k.push_back({"row_radix", &pss_system::tune_row_radix, {8, 16}});
        if (s->dim == 3) {
            k.push_back({"mid_radix", &pss_system::tune_mid_radix, {8, 16}});
            k.push_back({"mid_planes", &pss_system::tune_mid_planes, {1, 2, 4}});
        }
        if (!fast3d_rows(s)) k.push_back({"row_pairs", &pss_system::tune_row_pairs, {1, 2, 4, 8}});
        k.push_back({"col_tiles", &pss_system::tune_col_tiles, {1, 2, 4}});
    }
    k.push_back({"pdl", &pss_system::tune_pdl, {0, 1}});
    k.push_back({"graph_steps", &pss_system::tune_graph_steps, {8, 16, 32}});
    return k;
}

// Milliseconds per step: the fastest of `reps` timed runs of at least `n`
// steps (a whole number of graph replays), after one replay of warm-up that
// also captures the graph of the current launch shape.
int tune_trial(pss_system *s, int64_t n, int reps, cudaEvent_t e0, cudaEvent_t e1, double *ms) {
    const int chunk = s->tune_graph_steps > 0 ? s->tune_graph_steps : kDefaultGraphSteps;
    const int64_t m = (n + chunk - 1) / chunk * chunk;
    int rc = pss_step(s, chunk);
    if (rc) return rc;
    double best = 1e300;
    for (int r = 0; r < reps; ++r) {
        CK(cudaEventRecord(e0, s->stream));
        if ((rc = pss_step(s, m))) return rc;
        CK(cudaEventRecord(e1, s->stream));
        CK(cudaEventSynchronize(e1));
        float t = 0;
        CK(cudaEventElapsedTime(&t, e0, e1));
        best = std::min(best, (double)t / (double)m);
    }
    *ms = best;
    return PSS_OK;
}

int autotune_search(pss_system *s, int64_t n, const std::vector<TuneKnob> &space, const std::vector<int> &initial,
                    double *ms_initial, double *ms_tuned, int *trials, int *skipped) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) { cudaEventDestroy(e0); return cuda_fail(s, ce, "cudaEventCreate"); }
    const int reps = 3;
    int rc = PSS_OK;
    double best = 0;
    *trials = 0;
    *skipped = 0;
    if ((rc = tune_trial(s, n, reps, e0, e1, &best)) == PSS_OK) {
        ++*trials;
        for (const TuneKnob &k : space) {
            const int keep = s->*k.field;
            int arg = keep;
            for (int v : k.values) {
                if (v == keep) continue;
                s->*k.field = v;
                invalidate(s);
                double t = 0;
                const int trc = tune_trial(s, n, reps, e0, e1, &t);
                if (trc) {
                    // a shape the launcher refuses for this system (its shared memory
                    // would not fit): skip it, as long as the stream is unharmed
                    cudaGetLastError();
                    if (cudaStreamSynchronize(s->stream) != cudaSuccess) { rc = trc; break; }
                    ++*skipped;
                    continue;
                }
                ++*trials;
                if (t < 0.99 * best) { best = t; arg = v; }
            }
            s->*k.field = arg;
            invalidate(s);
            if (rc) break;
        }
    }
    // the starting shape and the result, timed back to back twice over; the
    // result stands only if it is faster there too
    std::vector<int> tuned(space.size());
    for (size_t i = 0; i < space.size(); ++i) tuned[i] = s->*space[i].field;
    double t_init = 1e300, t_tuned = 1e300;
    for (int round = 0; round < 2 && rc == PSS_OK; ++round)
        for (int which = 0; which < 2 && rc == PSS_OK; ++which) {
            const std::vector<int> &set = which == 0 ? initial : tuned;
            for (size_t i = 0; i < space.size(); ++i) s->*space[i].field = set[i];
            invalidate(s);
            double t = 0;
            if ((rc = tune_trial(s, n, reps, e0, e1, &t))) break;
            ++*trials;
            (which == 0 ? t_init : t_tuned) = std::min(which == 0 ? t_init : t_tuned, t);
        }
    const std::vector<int> &final_set = (rc == PSS_OK && t_tuned <= t_init) ? tuned : initial;
    for (size_t i = 0; i < space.size(); ++i) s->*space[i].field = final_set[i];
    invalidate(s);
    *ms_initial = t_init;
    *ms_tuned = std::min(t_init, t_tuned);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

}  // namespace

extern "C" {

int pss_autotune(pss_system *s, int64_t steps_per_trial, char *report, size_t report_len) {
    if (!s) return PSS_EINVAL;
    if (steps_per_trial < 1) return fail(s, PSS_EINVAL, "steps_per_trial must be >= 1");
    if (s->fields.empty()) return fail(s, PSS_EINVAL, "no fields");
    if (report && report_len) report[0] = '\0';
    int rc = upload_params(s);
    if (rc) return rc;
    if (round_trip(s) && (rc = ensure_real(s))) return rc;
    if ((rc = prologue(s, persist2d(s)))) return rc;
    // keep the state and the step counter: the trials advance the system
    const size_t bytes = csize(s) * s->field_elems * (size_t)s->nslots();
    void *saved = nullptr;
    CK(cudaMalloc(&saved, bytes));
    const int64_t step0 = s->step;
    cudaError_t e = cudaMemcpyAsync(saved, s->state, bytes, cudaMemcpyDeviceToDevice, s->stream);
    if (e != cudaSuccess) { cudaFree(saved); return cuda_fail(s, e, "saving the state"); }

    const std::vector<TuneKnob> space = tune_space(s);
    std::vector<int> initial(space.size());
    for (size_t i = 0; i < space.size(); ++i) initial[i] = s->*space[i].field;
    double ms_init = 0, ms_tuned = 0;
    int trials = 0, skipped = 0;
    rc = autotune_search(s, steps_per_trial, space, initial, &ms_init, &ms_tuned, &trials, &skipped);
    const std::string search_err = s->err;

    // put the state, the step counter and the next step's product and noise back
    long long v = step0;
    e = cudaMemcpyAsync(s->state, saved, bytes, cudaMemcpyDeviceToDevice, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->d_step, &v, sizeof v, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    cudaFree(saved);
    s->step = step0;
    s->stale = true;
    invalidate(s);
    if (rc) { s->err = search_err; return rc; }
    if (e != cudaSuccess) return cuda_fail(s, e, "restoring the state");
    if ((rc = device_errors(s))) return rc;

    if (report && report_len) {
        std::string r;
        char buf[160];
        snprintf(buf, sizeof buf, "path=%d trials=%d skipped=%d initial_ms=%.6g tuned_ms=%.6g", pss_step_path(s), trials,
                 skipped, ms_init, ms_tuned);
        r = buf;
        for (size_t i = 0; i < space.size(); ++i) {
            snprintf(buf, sizeof buf, " %s=%d", space[i].name, s->*space[i].field);
            r += buf;
        }
        snprintf(report, report_len, "%s", r.c_str());
    }
    return PSS_OK;
}

int pss_get_step(pss_system *s, int64_t *step) {
    if (!s || !step) return PSS_EINVAL;
    *step = s->step;
    return PSS_OK;
}

int pss_set_step(pss_system *s, int64_t step) {
    if (!s) return PSS_EINVAL;
    if (step < 0) return fail(s, PSS_EINVAL, "step must be >= 0");
    long long v = step;
    CK(cudaMemcpyAsync(s->d_step, &v, sizeof v, cudaMemcpyHostToDevice, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    s->step = step;
    s->stale = true;   // the fast 2D path keeps the next step's noise drawn ahead
    return PSS_OK;
}

int pss_get_field(pss_system *s, int field_id, void *real_out, int where) {
    int rc = check_field(s, field_id);
    if (rc) return rc;
    if (!real_out) return fail(s, PSS_EINVAL, "real_out is NULL");
    if ((rc = ensure_real(s))) return rc;
    if ((rc = upload_params(s))) return rc;
    const int slot = cur_slot(s, field_id);
    rc = s->prec == PSS_F64 ? inverse_slot<double>(s, slot) : inverse_slot<float>(s, slot);
    if (rc) return rc;
    if (s->dim == 3) s->stale = true;   // the y pass reused B
    const size_t bytes = rsize(s) * (size_t)s->nsites;
    CK(cudaMemcpyAsync(real_out, s->real, bytes, where == PSS_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                       s->stream));
    return device_errors(s);
}

int pss_get_spectrum(pss_system *s, int field_id, void *half_out, int where) {
    int rc = check_field(s, field_id);
    if (rc) return rc;
    if (!half_out) return fail(s, PSS_EINVAL, "half_out is NULL");
    if ((rc = ensure_half(s))) return rc;
    const size_t ofs = csize(s) * s->field_elems * (size_t)cur_slot(s, field_id);
    cudaError_t e = s->prec == PSS_F64
        ? launch_tiles_to_half<double>(sys_params<double>(s), (const double2 *)((char *)s->state + ofs),
                                       (double2 *)s->half, s->stream)
        : launch_tiles_to_half<float>(sys_params<float>(s), (const float2 *)((char *)s->state + ofs), (float2 *)s->half,
                                      s->stream);
    s->launches++;
    if (e != cudaSuccess) return cuda_fail(s, e, "layout kernel");
    const size_t bytes = csize(s) * (size_t)s->hx * s->ny * s->nz;
    CK(cudaMemcpyAsync(half_out, s->half, bytes, where == PSS_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                       s->stream));
    return device_errors(s);
}

int pss_set_spectrum(pss_system *s, int field_id, const void *half_in, int where) {
    int rc = check_field(s, field_id);
    if (rc) return rc;
    if (!half_in) return fail(s, PSS_EINVAL, "half_in is NULL");
    if ((rc = ensure_half(s))) return rc;
    const size_t bytes = csize(s) * (size_t)s->hx * s->ny * s->nz;
    CK(cudaMemcpyAsync(s->half, half_in, bytes, where == PSS_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                       s->stream));
    const size_t ofs = csize(s) * s->field_elems * (size_t)cur_slot(s, field_id);
    cudaError_t e = s->prec == PSS_F64
        ? launch_half_to_tiles<double>(sys_params<double>(s), (const double2 *)s->half,
                                       (double2 *)((char *)s->state + ofs), s->stream)
        : launch_half_to_tiles<float>(sys_params<float>(s), (const float2 *)s->half, (float2 *)((char *)s->state + ofs),
                                      s->stream);
    s->launches++;
    if (e != cudaSuccess) return cuda_fail(s, e, "layout kernel");
    s->stale = true;
    return PSS_OK;
}

// ---- checkpoint / resume -------------------------------------------------
// The saved state is everything a step reads that the caller can change:
// the half spectra of every field of every instance (in the exchange layout
// [nz][ny][nx/2+1], independent of the device layout), the step counter (the
// next step's noise index), the parameter values of every instance and the
// per-instance seeds.  The next step's product and drawn-ahead noise are not
// saved: both are functions of the state and the step counter, recomputed
// before the first step after a load.
namespace {
struct StateHeader {
    char magic[8];
    uint32_t version, header_bytes;
    int32_t dim, nx, ny, nz, precision, batch, nfields, nparams;
    int64_t step;
    uint64_t payload_bytes;
};
constexpr char kStateMagic[8] = {'P', 'S', 'S', 'S', 'T', 'A', 'T', 'E'};

size_t state_payload(const pss_system *s) {
    const size_t half = csize(s) * (size_t)s->hx * s->ny * s->nz;
    return sizeof(double) * (size_t)s->batch * s->param_names.size() + sizeof(uint64_t) * (size_t)s->batch +
           half * (size_t)s->nslots();
}
}  // namespace

int pss_save_state(pss_system *s, void *buf, size_t *len) {
    if (!s || !len) return PSS_EINVAL;
    if (s->fields.empty()) return fail(s, PSS_EINVAL, "no fields");
    const size_t need = sizeof(StateHeader) + state_payload(s);
    if (!buf) {
        *len = need;
        return PSS_OK;
    }
    if (*len < need) {
        *len = need;
        return fail(s, PSS_EINVAL, "buffer too small: %zu bytes needed", need);
    }
    int rc = ensure_half(s);
    if (rc) return rc;
    StateHeader h{};
    std::memcpy(h.magic, kStateMagic, 8);
    h.version = 1;
    h.header_bytes = sizeof(StateHeader);
    h.dim = s->dim; h.nx = s->nx; h.ny = s->ny; h.nz = s->nz;
    h.precision = s->prec;
    h.batch = s->batch;
    h.nfields = (int)s->fields.size();
    h.nparams = (int)s->param_names.size();
    h.step = s->step;
    h.payload_bytes = state_payload(s);
    char *p = (char *)buf;
    std::memcpy(p, &h, sizeof h);
    p += sizeof h;
    const size_t pv = sizeof(double) * s->param_values.size();
    if (pv) std::memcpy(p, s->param_values.data(), pv);
    p += pv;
    std::memcpy(p, s->seeds.data(), sizeof(uint64_t) * (size_t)s->batch);
    p += sizeof(uint64_t) * (size_t)s->batch;
    const size_t half = csize(s) * (size_t)s->hx * s->ny * s->nz;
    for (int slot = 0; slot < s->nslots(); ++slot, p += half) {
        const size_t ofs = csize(s) * s->field_elems * (size_t)slot;
        cudaError_t e = s->prec == PSS_F64
            ? launch_tiles_to_half<double>(sys_params<double>(s), (const double2 *)((char *)s->state + ofs),
                                           (double2 *)s->half, s->stream)
            : launch_tiles_to_half<float>(sys_params<float>(s), (const float2 *)((char *)s->state + ofs),
                                          (float2 *)s->half, s->stream);
        s->launches++;
        if (e != cudaSuccess) return cuda_fail(s, e, "layout kernel");
        CK(cudaMemcpyAsync(p, s->half, half, cudaMemcpyDeviceToHost, s->stream));
        CK(cudaStreamSynchronize(s->stream));   // s->half is reused by the next slot
    }
    *len = need;
    return device_errors(s);
}

int pss_load_state(pss_system *s, const void *buf, size_t len) {
    if (!s || !buf) return PSS_EINVAL;
    if (s->fields.empty()) return fail(s, PSS_EINVAL, "no fields");
    StateHeader h{};
    if (len < sizeof h) return fail(s, PSS_EINVAL, "not a saved state: %zu bytes", len);
    std::memcpy(&h, buf, sizeof h);
    if (std::memcmp(h.magic, kStateMagic, 8) != 0 || h.version != 1 || h.header_bytes != sizeof h)
        return fail(s, PSS_EINVAL, "not a saved state of this format");
    if (h.dim != s->dim || h.nx != s->nx || h.ny != s->ny || h.nz != s->nz || h.precision != s->prec ||
        h.batch != s->batch || h.nfields != (int)s->fields.size() || h.nparams != (int)s->param_names.size())
        return fail(s, PSS_EINVAL,
                    "saved state of a different system (dim %d, %dx%dx%d, precision %d, batch %d, %d fields, "
                    "%d parameters)", h.dim, h.nx, h.ny, h.nz, h.precision, h.batch, h.nfields, h.nparams);
    if (h.payload_bytes != state_payload(s) || len < sizeof h + h.payload_bytes || h.step < 0)
        return fail(s, PSS_EINVAL, "saved state is truncated or inconsistent");
    int rc = ensure_half(s);
    if (rc) return rc;
    const char *p = (const char *)buf + sizeof h;
    const size_t pv = sizeof(double) * s->param_values.size();
    if (pv) std::memcpy(s->param_values.data(), p, pv);
    p += pv;
    std::memcpy(s->seeds.data(), p, sizeof(uint64_t) * (size_t)s->batch);
    p += sizeof(uint64_t) * (size_t)s->batch;
    s->fps_dirty = true;
    const size_t half = csize(s) * (size_t)s->hx * s->ny * s->nz;
    for (int slot = 0; slot < s->nslots(); ++slot, p += half) {
        CK(cudaMemcpyAsync(s->half, p, half, cudaMemcpyHostToDevice, s->stream));
        const size_t ofs = csize(s) * s->field_elems * (size_t)slot;
        cudaError_t e = s->prec == PSS_F64
            ? launch_half_to_tiles<double>(sys_params<double>(s), (const double2 *)s->half,
                                           (double2 *)((char *)s->state + ofs), s->stream)
            : launch_half_to_tiles<float>(sys_params<float>(s), (const float2 *)s->half,
                                          (float2 *)((char *)s->state + ofs), s->stream);
        s->launches++;
        if (e != cudaSuccess) return cuda_fail(s, e, "layout kernel");
        CK(cudaStreamSynchronize(s->stream));   // the host buffer and s->half are reused
    }
    long long v = h.step;
    CK(cudaMemcpyAsync(s->d_step, &v, sizeof v, cudaMemcpyHostToDevice, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    s->step = h.step;
    s->stale = true;   // the next step's product and noise come from the loaded state
    if (!s->gterms.empty()) invalidate(s);   // product-term operators are launch arguments
    return device_errors(s);
}

int pss_structure_factor(pss_system *s, int field_id, int nbins, double *S_out, double *count_out, double *L_out) {
    int rc = check_field(s, field_id);
    if (rc) return rc;
    if (nbins < 1 || nbins > 4096 || !S_out) return fail(s, PSS_EINVAL, "nbins in [1, 4096] and S_out required");
    const int need = 2 * nbins + 2;
    if (s->sq_cap < need) {
        cudaFree(s->sq);
        s->sq = nullptr;
        s->sq_cap = 0;   // a failed allocation below leaves no capacity behind
        CK(cudaMalloc(&s->sq, sizeof(double) * need));
        s->sq_cap = need;
    }
    CK(cudaMemsetAsync(s->sq, 0, sizeof(double) * need, s->stream));
    const size_t ofs = csize(s) * s->field_elems * (size_t)cur_slot(s, field_id);
    cudaError_t e = s->prec == PSS_F64
        ? launch_structure_factor<double>(sys_params<double>(s), s->dx, (const double2 *)((char *)s->state + ofs), nbins,
                                          s->sq, s->stream)
        : launch_structure_factor<float>(sys_params<float>(s), s->dx, (const float2 *)((char *)s->state + ofs), nbins,
                                         s->sq, s->stream);
    s->launches++;
    if (e != cudaSuccess) return cuda_fail(s, e, "structure factor kernel");
    std::vector<double> h(need);
    CK(cudaMemcpyAsync(h.data(), s->sq, sizeof(double) * need, cudaMemcpyDeviceToHost, s->stream));
    if ((rc = device_errors(s))) return rc;
    for (int b = 0; b < nbins; ++b) {
        S_out[b] = h[nbins + b] > 0 ? h[b] / h[nbins + b] : 0.0;
        if (count_out) count_out[b] = h[nbins + b];
    }
    if (L_out) *L_out = h[2 * nbins + 1] > 0 ? 2 * kPi * h[2 * nbins] / h[2 * nbins + 1] : 0.0;
    return PSS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Structure factor without allocation.  The bin accumulator is a fixed array
// of this file; host code reaches it only through the device address that
// cudaGetSymbolAddress returns (the name itself, in host code, is a host-side
// stand-in and must never be handed to a kernel).
// ---------------------------------------------------------------------------
namespace {
constexpr int kNoAllocSlots = 2 * PSS_NOALLOC_MAX_BINS + 2;   // bin sums, bin counts, two totals
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) double g_sq_scratch[kNoAllocSlots];

std::mutex g_sq_setup_mutex;
double *g_sq_scratch_addr[kNoAllocMaxDevices];   // device address of g_sq_scratch, per device, once set up
}  // namespace

extern "C" {

int pss_structure_factor_noalloc(pss_system *s, int field_id, int nbins, double *S_out, double *count_out,
                                 double *L_out) {
    int rc = check_field(s, field_id);
    if (rc) return rc;
    if (nbins < 1 || nbins > PSS_NOALLOC_MAX_BINS || !S_out)
        return fail(s, PSS_EINVAL, "nbins in [1, PSS_NOALLOC_MAX_BINS = %d] and S_out required",
                    PSS_NOALLOC_MAX_BINS);
    int dev = -1;
    CK(cudaGetDevice(&dev));
    if (dev != s->device) return fail(s, PSS_EINVAL, "the system's device (%d) is not the current device", s->device);
    if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(s, PSS_EUNSUPPORTED, "device index %d too large", dev);
    double *acc = nullptr;
    {
        // set-up, once per device, with that device current
        std::lock_guard<std::mutex> lock(g_sq_setup_mutex);
        if (!g_sq_scratch_addr[dev]) {
            void *addr = nullptr;
            cudaError_t e = cudaGetSymbolAddress((void **)&addr, g_sq_scratch);
            if (e != cudaSuccess) return cuda_fail(s, e, "cudaGetSymbolAddress of the structure-factor array");
            g_sq_scratch_addr[dev] = (double *)addr;
        }
        acc = g_sq_scratch_addr[dev];
    }
    const int need = 2 * nbins + 2;
    // the array keeps the previous call's sums: clear the part this call accumulates into
    CK(cudaMemsetAsync(acc, 0, sizeof(double) * need, s->stream));
    const size_t ofs = csize(s) * s->field_elems * (size_t)cur_slot(s, field_id);
    cudaError_t e = s->prec == PSS_F64
        ? launch_structure_factor<double>(sys_params<double>(s), s->dx, (const double2 *)((char *)s->state + ofs), nbins,
                                          acc, s->stream)
        : launch_structure_factor<float>(sys_params<float>(s), s->dx, (const float2 *)((char *)s->state + ofs), nbins,
                                         acc, s->stream);
    s->launches++;
    if (e != cudaSuccess) return cuda_fail(s, e, "structure factor kernel");
    double h[kNoAllocSlots];   // host copy on the stack: no heap allocation either
    CK(cudaMemcpyAsync(h, acc, sizeof(double) * need, cudaMemcpyDeviceToHost, s->stream));
    if ((rc = device_errors(s))) return rc;
    for (int b = 0; b < nbins; ++b) {
        S_out[b] = h[nbins + b] > 0 ? h[b] / h[nbins + b] : 0.0;
        if (count_out) count_out[b] = h[nbins + b];
    }
    if (L_out) *L_out = h[2 * nbins + 1] > 0 ? 2 * kPi * h[2 * nbins] / h[2 * nbins + 1] : 0.0;
    return PSS_OK;
}

int pss_sync(pss_system *s) {
    if (!s) return PSS_EINVAL;
    return device_errors(s);
}

const char *pss_last_error(const pss_system *s) { return s ? s->err.c_str() : g_create_err.c_str(); }

int64_t pss_launch_count(const pss_system *s) { return s ? s->launches : 0; }

int pss_step_path(const pss_system *s) {
    return s ? (persist2d(s) ? 3 : fast2d(s) ? 1 : fast3d_rows(s) ? 2 : 0) : PSS_EINVAL;
}

}  // extern "C"

"""Thin ctypes binding of libpss (include/pss.h).

Every method marshals arguments and calls the C function of the same name
(``pss_<method>``); all numerical work runs in the library's sm_103a kernels.
Host arrays are numpy; device arrays are torch CUDA tensors (their raw pointers
are passed with where=PSS_DEVICE).  There is no CPU fallback: if the library
is missing, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Iterable, Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(HERE, "_lib", "libpss.so")

PSS_OK, PSS_EINVAL, PSS_ENOMEM, PSS_ECUDA, PSS_ETIMEOUT, PSS_ENONFINITE, PSS_EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
PSS_F32, PSS_F64 = 0, 1
PSS_HOST, PSS_DEVICE = 0, 1
NOALLOC_MAX_BINS = 1024   # PSS_NOALLOC_MAX_BINS of the C header

EXPORTS = [
    "pss_create_system", "pss_destroy_system", "pss_set_stream", "pss_add_param", "pss_set_param",
    "pss_get_param", "pss_add_field", "pss_add_term", "pss_set_noise", "pss_set_dealias", "pss_set_field",
    "pss_init_uniform", "pss_step", "pss_get_step", "pss_set_step", "pss_get_field", "pss_get_spectrum",
    "pss_set_spectrum", "pss_structure_factor", "pss_sync", "pss_last_error", "pss_launch_count",
    "pss_time_kernels", "pss_set_tuning", "pss_create_batch", "pss_batch_size", "pss_select_instance",
    "pss_set_param_batch", "pss_step_many", "pss_adjoint_forward", "pss_adjoint_backward",
    "pss_structure_factor_noalloc", "pss_step_path", "pss_set_frame", "pss_add_grad_sq_term",
    "pss_add_product_term", "pss_autotune", "pss_save_state", "pss_load_state",
]


class PssError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libpss error {code}: {msg}")
        self.code = code


def _load():
    if not os.path.exists(LIBPATH):
        raise ImportError(f"{LIBPATH} is missing: build it with paper_2405_02410_gb300.build.build()")
    L = ctypes.CDLL(LIBPATH)
    vp, i32, i64, d, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_uint64
    P = ctypes.POINTER
    sig = {
        "pss_create_system": ([P(vp), i32, i32, i32, i32, d, d, d, d, u64, i32], i32),
        "pss_destroy_system": ([vp], i32),
        "pss_set_stream": ([vp, vp], i32),
        "pss_add_param": ([vp, ctypes.c_char_p, d, P(i32)], i32),
        "pss_set_param": ([vp, i32, d], i32),
        "pss_get_param": ([vp, i32, P(d)], i32),
        "pss_add_field": ([vp, ctypes.c_char_p, i32, P(i32)], i32),
        "pss_add_term": ([vp, i32, i32, i32, P(i32), P(d), P(i32), i32, P(i32), P(i32)], i32),
        "pss_add_grad_sq_term": ([vp, i32, i32, P(i32), P(d), P(i32)], i32),
        "pss_add_product_term": ([vp, i32, i32, P(i32), P(d), P(i32), i32, P(i32), P(i32), P(i32), P(i32)], i32),
        "pss_set_noise": ([vp, i32, i32, i32], i32),
        "pss_set_dealias": ([vp, i32, i32], i32),
        "pss_set_frame": ([vp, i32, i32, d, d], i32),
        "pss_set_field": ([vp, i32, vp, i32], i32),
        "pss_init_uniform": ([vp, i32, d, d], i32),
        "pss_step": ([vp, i64], i32),
        "pss_get_step": ([vp, P(i64)], i32),
        "pss_set_step": ([vp, i64], i32),
        "pss_get_field": ([vp, i32, vp, i32], i32),
        "pss_get_spectrum": ([vp, i32, vp, i32], i32),
        "pss_set_spectrum": ([vp, i32, vp, i32], i32),
        "pss_structure_factor": ([vp, i32, i32, P(d), P(d), P(d)], i32),
        "pss_structure_factor_noalloc": ([vp, i32, i32, P(d), P(d), P(d)], i32),
        "pss_sync": ([vp], i32),
        "pss_last_error": ([vp], ctypes.c_char_p),
        "pss_launch_count": ([vp], i64),
        "pss_step_path": ([vp], i32),
        "pss_time_kernels": ([vp, i64, P(d)], i32),
        "pss_set_tuning": ([vp, ctypes.c_char_p, i32], i32),
        "pss_autotune": ([vp, i64, ctypes.c_char_p, ctypes.c_size_t], i32),
        "pss_create_batch": ([P(vp), i32, i32, i32, i32, i32, d, d, d, d, P(u64), i32], i32),
        "pss_batch_size": ([vp], i32),
        "pss_select_instance": ([vp, i32], i32),
        "pss_set_param_batch": ([vp, i32, P(d)], i32),
        "pss_step_many": ([P(vp), i32, i64], i32),
        "pss_adjoint_forward": ([vp, i64], i32),
        "pss_adjoint_backward": ([vp, vp, i32, P(d), vp, i32], i32),
        "pss_save_state": ([vp, vp, P(ctypes.c_size_t)], i32),
        "pss_load_state": ([vp, vp, ctypes.c_size_t], i32),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    return L


lib = _load()


def _arr(ctype, vals):
    vals = list(vals)
    return (ctype * max(1, len(vals)))(*vals)


class System:
    """One lattice system (pss_create_system / pss_create_batch): ``System(shape, dt, dx, seed,
    precision, batch, seeds)``; shape is (nx,), (ny, nx) or (nz, ny, nx) like numpy arrays of the
    real field; batch > 1 (or seeds) makes independent instances keyed by seeds[i] (default seed + i)."""

    def __init__(self, shape: Sequence[int], dt: float, dx: Sequence[float] = (1.0, 1.0, 1.0),
                 seed: int = 0, precision: str = "f32", batch: int = 1, seeds: Optional[Sequence[int]] = None):
        self.shape = tuple(int(n) for n in shape)
        self.dim = len(self.shape)
        n = list(reversed(self.shape)) + [1] * (3 - self.dim)
        self.nx, self.ny, self.nz = n
        self.precision = precision
        self.rdtype = np.float64 if precision == "f64" else np.float32
        self.cdtype = np.complex128 if precision == "f64" else np.complex64
        h = ctypes.c_void_p()
        dxs = list(dx) + [1.0] * (3 - len(dx))
        prec = PSS_F64 if precision == "f64" else PSS_F32
        self.batch = int(batch)
        if self.batch == 1 and seeds is None:
            rc = lib.pss_create_system(ctypes.byref(h), self.dim, self.nx, self.ny, self.nz, dxs[0], dxs[1], dxs[2],
                                       float(dt), ctypes.c_uint64(int(seed) & 0xFFFFFFFFFFFFFFFF), prec)
        else:
            sd = list(seeds) if seeds is not None else [int(seed) + i for i in range(self.batch)]
            assert len(sd) == self.batch
            arr = (ctypes.c_uint64 * self.batch)(*[int(x) & 0xFFFFFFFFFFFFFFFF for x in sd])
            rc = lib.pss_create_batch(ctypes.byref(h), self.batch, self.dim, self.nx, self.ny, self.nz, dxs[0],
                                      dxs[1], dxs[2], float(dt), arr, prec)
        if rc != PSS_OK:
            raise PssError(rc, lib.pss_last_error(None).decode())
        self._h = h
        self.half_shape = self.shape[:-1] + (self.nx // 2 + 1,)

    # -- lifetime ------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            lib.pss_destroy_system(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ck(self, rc: int):
        if rc != PSS_OK:
            raise PssError(rc, lib.pss_last_error(self._h).decode())

    # -- model description ---------------------------------------------------
    def set_stream(self, stream=None):
        """stream: a torch.cuda.Stream, a raw cudaStream_t int, or None (legacy default)."""
        ptr = getattr(stream, "cuda_stream", stream)
        self._ck(lib.pss_set_stream(self._h, ctypes.c_void_p(ptr or 0)))

    def add_param(self, name: str, value: float) -> int:
        i = ctypes.c_int()
        self._ck(lib.pss_add_param(self._h, name.encode(), float(value), ctypes.byref(i)))
        self._param_names = getattr(self, "_param_names", []) + [name]
        return i.value

    def set_param(self, pid: int, value: float):
        self._ck(lib.pss_set_param(self._h, pid, float(value)))

    def set_param_batch(self, pid: int, values):
        v = np.ascontiguousarray(values, dtype=np.float64)
        assert v.shape == (self.batch,)
        self._ck(lib.pss_set_param_batch(self._h, pid, v.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))

    def select_instance(self, instance: int):
        self._ck(lib.pss_select_instance(self._h, int(instance)))

    def get_param(self, pid: int) -> float:
        v = ctypes.c_double()
        self._ck(lib.pss_get_param(self._h, pid, ctypes.byref(v)))
        return v.value

    def add_field(self, name: str, dynamic: bool = True) -> int:
        i = ctypes.c_int()
        self._ck(lib.pss_add_field(self._h, name.encode(), int(dynamic), ctypes.byref(i)))
        return i.value

    def add_term(self, field: int, implicit: bool, monomials: Iterable, factors: Iterable):
        """monomials: (param_id or -1, scale, q2_power); factors: (field_id, power)."""
        mono = list(monomials)
        fac = list(factors)
        self._ck(lib.pss_add_term(self._h, field, int(implicit), len(mono),
                                  _arr(ctypes.c_int, [m[0] for m in mono]),
                                  _arr(ctypes.c_double, [float(m[1]) for m in mono]),
                                  _arr(ctypes.c_int, [m[2] for m in mono]), len(fac),
                                  _arr(ctypes.c_int, [f[0] for f in fac]), _arr(ctypes.c_int, [f[1] for f in fac])))

    def add_grad_sq_term(self, field: int, monomials: Iterable):
        """rhs term M(q) F[|grad(m phi)|^2]; monomials: (param_id or -1, scale, q2_power)."""
        mono = list(monomials)
        self._ck(lib.pss_add_grad_sq_term(self._h, field, len(mono),
                                          _arr(ctypes.c_int, [m[0] for m in mono]),
                                          _arr(ctypes.c_double, [float(m[1]) for m in mono]),
                                          _arr(ctypes.c_int, [int(m[2]) for m in mono])))

    def add_product_term(self, field: int, monomials: Iterable, factors: Iterable):
        """rhs term M(q) F[prod_k psi_k^n_k]; monomials: (param_id or -1, scale, q2_power);
        factors: (field_id, power[, deriv axis or -1[, laplacian power]])."""
        mono = list(monomials)
        fac = [tuple(f) + (-1, 0)[len(f) - 2:] if len(f) < 4 else tuple(f) for f in factors]
        self._ck(lib.pss_add_product_term(self._h, field, len(mono),
                                          _arr(ctypes.c_int, [m[0] for m in mono]),
                                          _arr(ctypes.c_double, [float(m[1]) for m in mono]),
                                          _arr(ctypes.c_int, [int(m[2]) for m in mono]),
                                          len(fac), _arr(ctypes.c_int, [f[0] for f in fac]),
                                          _arr(ctypes.c_int, [f[1] for f in fac]),
                                          _arr(ctypes.c_int, [f[2] for f in fac]),
                                          _arr(ctypes.c_int, [f[3] for f in fac])))

    def set_noise(self, field: int, D_param: int, q2_pow: int = 0):
        self._ck(lib.pss_set_noise(self._h, field, D_param, q2_pow))

    def set_dealias(self, field: int, order: int):
        self._ck(lib.pss_set_dealias(self._h, field, order))

    def set_frame(self, field: int, width: int, lo: float, hi: float):
        """Boundary frame along x: after every step x < width takes lo and x >= Nx - width takes hi."""
        self._ck(lib.pss_set_frame(self._h, field, width, float(lo), float(hi)))

    # -- data ----------------------------------------------------------------
    def set_field(self, field: int, data):
        if _is_cuda_tensor(data):
            assert data.is_contiguous() and tuple(data.shape) == self.shape
            self._ck(lib.pss_set_field(self._h, field, ctypes.c_void_p(data.data_ptr()), PSS_DEVICE))
        else:
            a = np.ascontiguousarray(data, dtype=self.rdtype).reshape(self.shape)
            self._ck(lib.pss_set_field(self._h, field, a.ctypes.data_as(ctypes.c_void_p), PSS_HOST))

    def init_uniform(self, field: int, lo: float, hi: float):
        self._ck(lib.pss_init_uniform(self._h, field, float(lo), float(hi)))

    def step(self, n: int = 1):
        self._ck(lib.pss_step(self._h, int(n)))

    def get_step(self) -> int:
        v = ctypes.c_int64()
        self._ck(lib.pss_get_step(self._h, ctypes.byref(v)))
        return v.value

    def set_step(self, step: int):
        self._ck(lib.pss_set_step(self._h, int(step)))

    def get_field(self, field: int, out=None):
        """Real field; into ``out`` (numpy or torch CUDA tensor) or a new numpy array."""
        if out is not None and _is_cuda_tensor(out):
            self._ck(lib.pss_get_field(self._h, field, ctypes.c_void_p(out.data_ptr()), PSS_DEVICE))
            return out
        a = np.empty(self.shape, dtype=self.rdtype) if out is None else out
        self._ck(lib.pss_get_field(self._h, field, a.ctypes.data_as(ctypes.c_void_p), PSS_HOST))
        return a

    def get_spectrum(self, field: int, out=None):
        if out is not None and _is_cuda_tensor(out):
            self._ck(lib.pss_get_spectrum(self._h, field, ctypes.c_void_p(out.data_ptr()), PSS_DEVICE))
            return out
        a = np.empty(self.half_shape, dtype=self.cdtype) if out is None else out
        self._ck(lib.pss_get_spectrum(self._h, field, a.ctypes.data_as(ctypes.c_void_p), PSS_HOST))
        return a

    def set_spectrum(self, field: int, half):
        if _is_cuda_tensor(half):
            self._ck(lib.pss_set_spectrum(self._h, field, ctypes.c_void_p(half.data_ptr()), PSS_DEVICE))
        else:
            a = np.ascontiguousarray(half, dtype=self.cdtype).reshape(self.half_shape)
            self._ck(lib.pss_set_spectrum(self._h, field, a.ctypes.data_as(ctypes.c_void_p), PSS_HOST))

    def save_state(self) -> bytes:
        """The whole state (spectra of every field and instance, step counter, parameters, seeds)
        as bytes (pss_save_state)."""
        n = ctypes.c_size_t(0)
        self._ck(lib.pss_save_state(self._h, None, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        self._ck(lib.pss_save_state(self._h, ctypes.cast(buf, ctypes.c_void_p), ctypes.byref(n)))
        return buf.raw[: n.value]

    def load_state(self, blob: bytes):
        """Restore a state written by save_state into a system built the same way (pss_load_state)."""
        buf = ctypes.create_string_buffer(bytes(blob), len(blob))
        self._ck(lib.pss_load_state(self._h, ctypes.cast(buf, ctypes.c_void_p), len(blob)))

    def structure_factor(self, field: int, nbins: int = 64):
        S = np.zeros(nbins)
        cnt = np.zeros(nbins)
        L = ctypes.c_double()
        dp = ctypes.POINTER(ctypes.c_double)
        self._ck(lib.pss_structure_factor(self._h, field, nbins, S.ctypes.data_as(dp), cnt.ctypes.data_as(dp),
                                          ctypes.byref(L)))
        return S, cnt, L.value

    def structure_factor_noalloc(self, field: int, nbins: int = 64):
        """structure_factor computed with the library's fixed accumulator (at most
        NOALLOC_MAX_BINS bins): the library allocates no memory for it, for callers
        that must not allocate while they run.  Calls that overlap on the GPU race."""
        S = np.zeros(nbins)
        cnt = np.zeros(nbins)
        L = ctypes.c_double()
        dp = ctypes.POINTER(ctypes.c_double)
        self._ck(lib.pss_structure_factor_noalloc(self._h, field, nbins, S.ctypes.data_as(dp),
                                                  cnt.ctypes.data_as(dp), ctypes.byref(L)))
        return S, cnt, L.value

    def time_kernels(self, n: int):
        """Mean per-launch milliseconds of (column, inverse-y, row, forward-y) kernels over n steps."""
        out = (ctypes.c_double * 4)()
        self._ck(lib.pss_time_kernels(self._h, int(n), out))
        return list(out)

    def set_tuning(self, key: str, value: int):
        """Launch-shape knob ("pdl", "row_pairs", "col_tiles", "mid_planes", "graph_steps", "col_radix",
        "row_radix", "mid_radix", "fast2d", "fast3d", "col2_warps", "row2_pairs", "row2_noise", "col2_radix",
        "row2_radix", "adj_row_pairs", ...; see pss_set_tuning in include/pss.h); 0 = automatic (for "fast2d" / "fast3d": the generic kernels)."""
        self._ck(lib.pss_set_tuning(self._h, key.encode(), int(value)))

    def autotune(self, steps_per_trial: int = 64) -> dict:
        """Time the launch-shape knobs of this system's step path on the GPU and keep the
        fastest settings (pss_autotune); the state and step counter are left as they were.
        Returns the report as a dict: path, trials, initial_ms / tuned_ms per step, and each
        knob's pss_set_tuning value (0 = automatic, -1 = automatic for "pdl")."""
        buf = ctypes.create_string_buffer(1024)
        self._ck(lib.pss_autotune(self._h, int(steps_per_trial), buf, len(buf)))
        return parse_tune_report(buf.value.decode())

    def set_tunings(self, report: dict):
        """Apply the knob settings of an autotune report (other keys are ignored)."""
        for key, val in report.items():
            if key in ("path", "trials", "skipped", "initial_ms", "tuned_ms") or (key == "pdl" and val < 0):
                continue
            self.set_tuning(key, val)

    def adjoint_forward(self, n: int):
        """Advance n steps keeping sqrt(n)-spaced checkpoints for adjoint_backward."""
        self._ck(lib.pss_adjoint_forward(self._h, int(n)))

    def adjoint_backward(self, lambda_T, n_params: int):
        """dJ/dphi_T (half spectrum) -> (dJ/dparams[n_params] numpy, dJ/dphi_0 half spectrum).
        lambda_T a numpy array: dJ/dphi_0 comes back as numpy; a torch CUDA tensor of the
        system's complex dtype (contiguous, used on the system's stream): it comes back as a
        new CUDA tensor, and the spectra never leave the device."""
        g = np.zeros(max(1, n_params))
        if _is_cuda_tensor(lambda_T):
            import torch
            assert lambda_T.is_contiguous() and tuple(lambda_T.shape) == self.half_shape
            assert lambda_T.dtype == (torch.complex128 if self.precision == "f64" else torch.complex64)
            out = torch.empty_like(lambda_T)
            self._ck(lib.pss_adjoint_backward(self._h, ctypes.c_void_p(lambda_T.data_ptr()), PSS_DEVICE,
                                              g.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                              ctypes.c_void_p(out.data_ptr()), PSS_DEVICE))
            return g[:n_params], out
        lam = np.ascontiguousarray(lambda_T, dtype=self.cdtype).reshape(self.half_shape)
        out = np.empty(self.half_shape, dtype=self.cdtype)
        self._ck(lib.pss_adjoint_backward(self._h, lam.ctypes.data_as(ctypes.c_void_p), PSS_HOST,
                                          g.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                          out.ctypes.data_as(ctypes.c_void_p), PSS_HOST))
        return g[:n_params], out

    def sync(self):
        self._ck(lib.pss_sync(self._h))

    @property
    def launch_count(self) -> int:
        return int(lib.pss_launch_count(self._h))

    @property
    def step_path(self) -> str:
        """'persist2d' (k2p_step: a run of steps in one persistent launch; square FP32 2D, sides
        256..1024, one field), 'fast2d' (k2_col, k2_row: FP32 2D, sides 256..1024), 'fast3d_rows'
        (k_col, k_mid and the FFT-group x pass k2_row: FP32 3D, x side 256..1024) or 'generic'
        (k_col, k_mid, k_row)."""
        return {1: "fast2d", 2: "fast3d_rows", 3: "persist2d"}.get(lib.pss_step_path(self._h), "generic")


def parse_tune_report(text: str) -> dict:
    """'path=1 trials=9 initial_ms=0.0153 tuned_ms=0.0151 pdl=-1 ...' -> dict (ints, and floats for *_ms)."""
    out = {}
    for item in text.split():
        key, _, val = item.partition("=")
        out[key] = float(val) if key.endswith("_ms") else int(val)
    return out


def step_many(systems: Sequence[System], n: int):
    """Advance several systems by n steps from one captured CUDA graph (on systems[0]'s stream)."""
    arr = (ctypes.c_void_p * len(systems))(*[s._h for s in systems])
    rc = lib.pss_step_many(arr, len(systems), int(n))
    if rc != PSS_OK:
        raise PssError(rc, lib.pss_last_error(systems[0]._h).decode())


def _is_cuda_tensor(x) -> bool:
    return hasattr(x, "is_cuda") and bool(getattr(x, "is_cuda"))


# ---------------------------------------------------------------------------
# model builders (section "Example": Model B; its non-conserved sibling Model A)
# ---------------------------------------------------------------------------
def model_b(shape, dt=0.01, a=-1.0, b=1.0, K=1.0, D=0.01, noisy=True, seed=2405, precision="f32",
            dealias_order=2, dx=(1.0, 1.0, 1.0), system: Optional[System] = None) -> System:
    """dt phi + (a q^2 + K q^4) phi = -b q^2 phi^3, noise D q^2."""
    s = system or System(shape, dt=dt, dx=dx, seed=seed, precision=precision)
    add_model_b_field(s, a=a, b=b, K=K, D=D, noisy=noisy, dealias_order=dealias_order)
    return s


def add_model_b_field(s: System, a=-1.0, b=1.0, K=1.0, D=0.01, noisy=True, dealias_order=2, name="phi"):
    f = s.add_field(name)
    pa, pb, pK, pD = (s.add_param(f"{name}.{k}", v) for k, v in (("a", a), ("b", b), ("K", K), ("D", D)))
    s.add_term(f, True, [(pa, 1.0, 1), (pK, 1.0, 2)], [(f, 1)])
    s.add_term(f, False, [(pb, -1.0, 1)], [(f, 3)])
    if noisy:
        s.set_noise(f, pD, 1)
    s.set_dealias(f, dealias_order)
    return f


def add_kpz_field(s: System, sigma=1.0, lam=1.0, D=0.01, noisy=True, dealias_order=2, name="h"):
    """KPZ (section "Writing models"): dt h = sigma lap h + lambda (grad h)^2 + noise D,
    i.e. dt h + sigma q^2 h = lambda F[|grad(m h)|^2]."""
    f = s.add_field(name)
    ps, pl, pD = (s.add_param(f"{name}.{k}", v) for k, v in (("sigma", sigma), ("lambda", lam), ("D", D)))
    s.add_term(f, True, [(ps, 1.0, 1)], [(f, 1)])
    s.add_grad_sq_term(f, [(pl, 1.0, 0)])
    if noisy:
        s.set_noise(f, pD, 0)
    s.set_dealias(f, dealias_order)
    return f


def kpz(shape, dt=0.01, sigma=1.0, lam=1.0, D=0.01, noisy=True, seed=2405, precision="f32", dealias_order=2,
        dx=(1.0, 1.0, 1.0), system: Optional[System] = None) -> System:
    s = system or System(shape, dt=dt, dx=dx, seed=seed, precision=precision)
    add_kpz_field(s, sigma=sigma, lam=lam, D=D, noisy=noisy, dealias_order=dealias_order)
    return s


def add_model_a_field(s: System, a=-1.0, b=1.0, K=1.0, D=0.05, noisy=True, dealias_order=2, name="psi"):
    """dt psi + (a + K q^2) psi = -b psi^3, noise D."""
    f = s.add_field(name)
    pa, pb, pK, pD = (s.add_param(f"{name}.{k}", v) for k, v in (("a", a), ("b", b), ("K", K), ("D", D)))
    s.add_term(f, True, [(pa, 1.0, 0), (pK, 1.0, 1)], [(f, 1)])
    s.add_term(f, False, [(pb, -1.0, 0)], [(f, 3)])
    if noisy:
        s.set_noise(f, pD, 0)
    s.set_dealias(f, dealias_order)
    return f

"""ctypes binding of the FP64 CPU oracle (``pss_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It imports nothing
from the CUDA package, and the CUDA package never imports it.

Array conventions: real fields are ``float64[Nz, Ny, Nx]`` (x fastest, unused
axes dropped); spectra are full ``complex128`` arrays of the same shape in
standard FFT order.  ``half()`` slices a full spectrum to the R2C half
``[..., :Nx//2 + 1]``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field
from typing import Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_LIBPATH = os.path.join(_LIBDIR, "liboracle.so")
_SRC = os.path.join(_HERE, "pss_oracle.c")
MAX_MONO = 8
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no fast-math, no FMA contraction)."""
    with _lock:
        if (not force and os.path.exists(_LIBPATH)
                and os.path.getmtime(_LIBPATH) >= os.path.getmtime(_SRC)
                and os.path.getmtime(_LIBPATH) >= os.path.getmtime(os.path.join(_HERE, "pss_oracle.h"))):
            return _LIBPATH
        os.makedirs(_LIBDIR, exist_ok=True)
        tmp = _LIBPATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIBPATH)
        return _LIBPATH


class _Field(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("n", ctypes.c_int * 3),
        ("dx", ctypes.c_double * 3),
        ("dt", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("field_id", ctypes.c_int),
        ("n_lhs", ctypes.c_int),
        ("lhs_coef", ctypes.c_double * MAX_MONO),
        ("lhs_pow", ctypes.c_int * MAX_MONO),
        ("n_rhs", ctypes.c_int),
        ("rhs_coef", ctypes.c_double * MAX_MONO),
        ("rhs_pow", ctypes.c_int * MAX_MONO),
        ("power", ctypes.c_int),
        ("noisy", ctypes.c_int),
        ("noise_D", ctypes.c_double),
        ("noise_pow", ctypes.c_int),
        ("dealias_order", ctypes.c_int),
        ("transform", ctypes.c_int),
        ("grad2", ctypes.c_int),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        d = P(ctypes.c_double)
        f = P(_Field)
        _lib.orc_philox4x32_10.argtypes = [P(ctypes.c_uint32), P(ctypes.c_uint32), P(ctypes.c_uint32)]
        _lib.orc_uniform24.argtypes = [ctypes.c_uint32]
        _lib.orc_uniform24.restype = ctypes.c_double
        _lib.orc_normal_pair.argtypes = [ctypes.c_uint64] + [ctypes.c_uint32] * 4 + [d, d]
        _lib.orc_normal_pair_words.argtypes = [ctypes.c_uint64] + [ctypes.c_uint32] * 4 + [ctypes.c_int, d, d]
        _lib.orc_dft.argtypes = [ctypes.c_int, P(ctypes.c_int), d, ctypes.c_int, ctypes.c_int]
        _lib.orc_mask.argtypes = [f, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        _lib.orc_q2.argtypes = [f, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        _lib.orc_q2.restype = ctypes.c_double
        _lib.orc_nonlinear.argtypes = [f, d, d]
        _lib.orc_noise.argtypes = [f, ctypes.c_int64, d]
        _lib.orc_run.argtypes = [f, d, ctypes.c_int64, ctypes.c_int64]
        _lib.orc_init_uniform.argtypes = [f, ctypes.c_double, ctypes.c_double, d]
        _lib.orc_structure_factor.argtypes = [f, d, ctypes.c_int, d, d, d]
        _lib.orc_adjoint.argtypes = [f, d, ctypes.c_int64, ctypes.c_int64, d, d]
    return _lib


def _dptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclass
class Model:
    """One dynamic field: ``dt phi + O(q) phi = M(q) F[(F^-1[m phi])^power]`` plus noise
    ``D~ = noise_D (q^2)^noise_pow``.  ``lhs``/``rhs`` are lists of ``(coef, q2_power)``."""

    shape: Sequence[int]                      # (Nx,), (Ny, Nx) or (Nz, Ny, Nx)
    dt: float
    lhs: list = field(default_factory=list)
    rhs: list = field(default_factory=list)
    power: int = 0
    noise_D: float = 0.0
    noise_pow: int = 0
    noisy: bool = False
    dealias_order: int = 2
    seed: int = 0
    field_id: int = 0
    dx: Sequence[float] = (1.0, 1.0, 1.0)     # (dx, dy, dz)
    transform: int = 0
    grad2: bool = False                       # product |grad(m phi)|^2 (KPZ) instead of (m phi)^power

    @property
    def dim(self) -> int:
        return len(self.shape)

    @property
    def n_sites(self) -> int:
        return int(np.prod(self.shape))

    def c_struct(self) -> _Field:
        s = _Field()
        s.dim = self.dim
        n = list(reversed(self.shape)) + [1] * (3 - self.dim)
        for j in range(3):
            s.n[j] = int(n[j])
            s.dx[j] = float(self.dx[j]) if j < self.dim else 1.0
        s.dt = float(self.dt)
        s.seed = int(self.seed) & 0xFFFFFFFFFFFFFFFF
        s.field_id = int(self.field_id)
        assert len(self.lhs) <= MAX_MONO and len(self.rhs) <= MAX_MONO
        s.n_lhs = len(self.lhs)
        for m, (c, p) in enumerate(self.lhs):
            s.lhs_coef[m] = float(c)
            s.lhs_pow[m] = int(p)
        s.n_rhs = len(self.rhs)
        for m, (c, p) in enumerate(self.rhs):
            s.rhs_coef[m] = float(c)
            s.rhs_pow[m] = int(p)
        s.power = int(self.power)
        s.noisy = int(bool(self.noisy))
        s.noise_D = float(self.noise_D)
        s.noise_pow = int(self.noise_pow)
        s.dealias_order = int(self.dealias_order)
        s.transform = int(self.transform)
        s.grad2 = int(bool(self.grad2))
        return s


def model_b(shape, dt=0.01, a=-1.0, b=1.0, K=1.0, D=0.01, noisy=True, seed=2405,
            dealias_order=2, field_id=0, dx=(1.0, 1.0, 1.0)) -> Model:
    """Model B / Cahn-Hilliard (section "Example"): dt phi + (a q^2 + K q^4) phi = -b q^2 phi^3,
    conserved noise D q^2."""
    return Model(shape=shape, dt=dt, lhs=[(a, 1), (K, 2)], rhs=[(-b, 1)], power=3,
                 noise_D=D, noise_pow=1, noisy=noisy, dealias_order=dealias_order,
                 seed=seed, field_id=field_id, dx=dx)


def kpz(shape, dt=0.01, sigma=1.0, lam=1.0, D=0.01, noisy=True, seed=2405, dealias_order=2, field_id=0,
        dx=(1.0, 1.0, 1.0)) -> Model:
    """KPZ (section "Writing models"): dt phi = sigma lap phi + lambda (grad phi)^2 + noise, i.e.
    dt phi + sigma q^2 phi = lambda F[|grad(m phi)|^2], non-conserved noise D (the quadratic
    term takes the two-thirds rule, order 2)."""
    return Model(shape=shape, dt=dt, lhs=[(sigma, 1)], rhs=[(lam, 0)], power=2, grad2=True,
                 noise_D=D, noise_pow=0, noisy=noisy, dealias_order=dealias_order,
                 seed=seed, field_id=field_id, dx=dx)


def model_a(shape, dt=0.005, a=-1.0, b=1.0, K=1.0, D=0.05, noisy=True, seed=2405,
            dealias_order=2, field_id=0, dx=(1.0, 1.0, 1.0)) -> Model:
    """Model A / Allen-Cahn: dt phi + (a + K q^2) phi = -b phi^3, noise strength D."""
    return Model(shape=shape, dt=dt, lhs=[(a, 0), (K, 1)], rhs=[(-b, 0)], power=3,
                 noise_D=D, noise_pow=0, noisy=noisy, dealias_order=dealias_order,
                 seed=seed, field_id=field_id, dx=dx)


# ---------------------------------------------------------------------------
# thin wrappers
# ---------------------------------------------------------------------------

def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 on arrays: ctr uint32[..., 4], key uint32[..., 2] -> uint32[..., 4]."""
    L = lib()
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(np.broadcast_to(np.asarray(key, dtype=np.uint32), (len(ctr), 2)))
    out = np.empty_like(ctr)
    P = ctypes.POINTER(ctypes.c_uint32)
    for i in range(len(ctr)):
        L.orc_philox4x32_10(ctr[i].ctypes.data_as(P), key[i].ctypes.data_as(P), out[i].ctypes.data_as(P))
    return out


def uniform24(x: int) -> float:
    return lib().orc_uniform24(ctypes.c_uint32(int(x)))


def normal_pair(seed, c0, c1, c2, c3):
    n1, n2 = ctypes.c_double(), ctypes.c_double()
    lib().orc_normal_pair(ctypes.c_uint64(int(seed)), c0, c1, c2, c3, ctypes.byref(n1), ctypes.byref(n2))
    return n1.value, n2.value


def normal_pair_words(seed, c0, c1, c2, c3, upper):
    n1, n2 = ctypes.c_double(), ctypes.c_double()
    lib().orc_normal_pair_words(ctypes.c_uint64(int(seed)), c0, c1, c2, c3, int(upper), ctypes.byref(n1),
                                ctypes.byref(n2))
    return n1.value, n2.value


def dft(x: np.ndarray, sign: int = -1, method: int = 2) -> np.ndarray:
    """Unnormalised d-dimensional DFT of a complex array (shape (Nx,), (Ny,Nx) or (Nz,Ny,Nx))."""
    a = np.ascontiguousarray(x, dtype=np.complex128).copy()
    dim = a.ndim
    n = (ctypes.c_int * 3)(*(list(reversed(a.shape)) + [1] * (3 - dim)))
    buf = a.view(np.float64)
    rc = lib().orc_dft(dim, n, _dptr(buf), int(sign), int(method))
    if rc:
        raise ValueError("orc_dft failed")
    return a


def mask(m: Model) -> np.ndarray:
    s = m.c_struct()
    N = list(reversed(m.shape)) + [1] * (3 - m.dim)
    out = np.zeros((N[2], N[1], N[0]), dtype=np.int32)
    for kz in range(N[2]):
        for ky in range(N[1]):
            for kx in range(N[0]):
                out[kz, ky, kx] = lib().orc_mask(ctypes.byref(s), kx, ky, kz)
    return out.reshape(m.shape)


def q2(m: Model) -> np.ndarray:
    s = m.c_struct()
    N = list(reversed(m.shape)) + [1] * (3 - m.dim)
    out = np.zeros((N[2], N[1], N[0]))
    for kz in range(N[2]):
        for ky in range(N[1]):
            for kx in range(N[0]):
                out[kz, ky, kx] = lib().orc_q2(ctypes.byref(s), kx, ky, kz)
    return out.reshape(m.shape)


def nonlinear(m: Model, phi: np.ndarray) -> np.ndarray:
    s = m.c_struct()
    phi = np.ascontiguousarray(phi, dtype=np.complex128)
    P = np.zeros_like(phi)
    if lib().orc_nonlinear(ctypes.byref(s), _dptr(phi.view(np.float64)), _dptr(P.view(np.float64))):
        raise ValueError("orc_nonlinear failed")
    return P


def noise(m: Model, step: int) -> np.ndarray:
    s = m.c_struct()
    xi = np.zeros(m.shape, dtype=np.complex128)
    lib().orc_noise(ctypes.byref(s), int(step), _dptr(xi.view(np.float64)))
    return xi


def run(m: Model, phi: np.ndarray, step0: int, nsteps: int) -> np.ndarray:
    """Return phi after ``nsteps`` steps (full spectrum, a new array)."""
    s = m.c_struct()
    out = np.ascontiguousarray(phi, dtype=np.complex128).copy()
    rc = lib().orc_run(ctypes.byref(s), _dptr(out.view(np.float64)), int(step0), int(nsteps))
    if rc:
        raise RuntimeError(f"orc_run failed ({rc})")
    return out


def run_framed(m: Model, phi: np.ndarray, step0: int, nsteps: int, width: int, lo: float, hi: float) -> np.ndarray:
    """``nsteps`` steps of Eq. timeupdate, each followed by a boundary frame
    (section "Callback functions"): the real field at the end of the step takes
    ``lo`` on the sites x < width and ``hi`` on the sites x >= Nx - width (every
    y and z), and the spectrum is taken again from that real field.
    ``width = 0`` is ``run``."""
    out = np.array(phi, dtype=np.complex128, copy=True)
    for k in range(nsteps):
        out = run(m, out, step0 + k, 1)
        if width > 0:
            r = to_real(m, out)
            r[..., :width] = lo
            r[..., r.shape[-1] - width:] = hi
            out = to_spectrum(m, r)
    return out


@dataclass
class Factor:
    """One factor psi^power of a product term, psi = F^-1[op(q) m phi_field] with
    op(q) = (i q_deriv if deriv >= 0) * (-q^2)^lap (section "Writing models": the
    fields psi_k are the fields phi_i acted on by differential operators)."""
    field: int
    power: int = 1
    deriv: int = -1           # -1: none; 0, 1, 2: i q_x, i q_y, i q_z (q = 0 at a Nyquist index)
    lap: int = 0


@dataclass
class Term:
    """M(q) F[prod_k psi_k^n_k] on the rhs of the equation of field ``target``;
    ``M`` is a list of (coef, q2_power)."""
    target: int
    M: list
    factors: list


def _q_axis(m: Model, axis: int) -> np.ndarray:
    """q_axis of every full-spectrum mode, 0 at a Nyquist index (odd operator)."""
    n = m.shape[m.dim - 1 - axis]
    k = np.arange(n)
    kk = np.where(k < (n + 1) // 2, k, k - n).astype(float)
    q = 2 * np.pi * kk / (n * m.dx[axis])
    if n % 2 == 0:
        q[n // 2] = 0.0
    shp = [1] * m.dim
    shp[m.dim - 1 - axis] = n
    return np.broadcast_to(q.reshape(shp), m.shape)


def term_products(models, terms, phis):
    """The explicit part P_i = sum_{terms of i} M_t(q) F[prod_k psi_k^n_k] of every
    field (Eq. basefourier with the nonlinearities written as in "Writing models"):
    each factor is taken to real space from its field's de-aliased spectrum, the
    factors multiply in real space, the product goes back to Fourier space."""
    m0 = models[0]
    method = 1 if m0.n_sites <= 256 else 2
    masks = [mask(m) for m in models]
    q2s = q2(m0)
    P = [np.zeros(m0.shape, dtype=np.complex128) for _ in models]
    for t in terms:
        prod = np.ones(m0.shape)
        for fct in t.factors:
            op = np.ones(m0.shape, dtype=np.complex128)
            if fct.deriv >= 0:
                op = op * 1j * _q_axis(m0, fct.deriv)
            op = op * (-q2s) ** fct.lap
            psi = dft(op * masks[fct.field] * phis[fct.field], +1, method).real / m0.n_sites
            prod = prod * psi ** fct.power
        Mq = sum(c * q2s ** p for c, p in t.M)
        P[t.target] = P[t.target] + Mq * dft(prod, -1, method)
    return P


def hermitian(phi: np.ndarray) -> np.ndarray:
    """The Hermitian part (phi_k + conj phi_-k) / 2 of a full spectrum."""
    flip = np.conj(np.roll(np.flip(phi), 1, axis=tuple(range(phi.ndim))))
    return 0.5 * (phi + flip)


def run_coupled(models, terms, phis, step0: int, nsteps: int):
    """Coupled fields (Eq. basefourier): every field i takes
    phi_i <- H[(phi_i + dt P_i + xi_i) / (1 + dt O_i(q))] with P_i from
    ``term_products`` of all fields at the same time step, O_i and the noise
    from ``models[i]`` (its own rhs and power are not used)."""
    phis = [np.array(p, dtype=np.complex128, copy=True) for p in phis]
    q2s = q2(models[0])
    for k in range(nsteps):
        P = term_products(models, terms, phis)
        nxt = []
        for i, m in enumerate(models):
            O = sum(c * q2s ** p for c, p in m.lhs) if m.lhs else np.zeros(m.shape)
            xi = noise(m, step0 + k) if m.noisy else 0.0
            nxt.append(hermitian((phis[i] + m.dt * P[i] + xi) / (1 + m.dt * O)))
        phis = nxt
    return phis


def init_uniform(m: Model, lo: float, hi: float) -> np.ndarray:
    s = m.c_struct()
    out = np.zeros(m.shape, dtype=np.float64)
    lib().orc_init_uniform(ctypes.byref(s), float(lo), float(hi), _dptr(out))
    return out


def to_spectrum(m: Model, real: np.ndarray) -> np.ndarray:
    return dft(np.asarray(real, dtype=np.complex128).reshape(m.shape), -1,
               1 if (m.transform == 1 or (m.transform == 0 and m.n_sites <= 256)) else 2)


def to_real(m: Model, phi: np.ndarray) -> np.ndarray:
    r = dft(phi, +1, 1 if (m.transform == 1 or (m.transform == 0 and m.n_sites <= 256)) else 2)
    return r.real / m.n_sites


def half(phi: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(phi[..., : phi.shape[-1] // 2 + 1])


def structure_factor(m: Model, phi: np.ndarray, nbins: int = 64):
    s = m.c_struct()
    phi = np.ascontiguousarray(phi, dtype=np.complex128)
    S = np.zeros(nbins)
    cnt = np.zeros(nbins)
    L = ctypes.c_double()
    lib().orc_structure_factor(ctypes.byref(s), _dptr(phi.view(np.float64)), int(nbins),
                               _dptr(S), _dptr(cnt), ctypes.byref(L))
    return S, cnt, L.value


def adjoint(m: Model, phi0: np.ndarray, step0: int, nsteps: int, lambda_T: np.ndarray):
    """Return (dJ/dphi_0, grad[11]) for dJ/dphi_T = lambda_T (full spectra; see orc_adjoint):
    grad[0:5] = dJ/dO_k, grad[5:10] = dJ/dM_k, grad[10] = dJ/dD."""
    s = m.c_struct()
    phi0 = np.ascontiguousarray(phi0, dtype=np.complex128)
    lam = np.ascontiguousarray(lambda_T, dtype=np.complex128).copy()
    g = np.zeros(11)
    rc = lib().orc_adjoint(ctypes.byref(s), _dptr(phi0.view(np.float64)), int(step0), int(nsteps),
                           _dptr(lam.view(np.float64)), _dptr(g))
    if rc:
        raise RuntimeError(f"orc_adjoint failed ({rc})")
    return lam, g


def binned_sq_loss(m: Model, phi: np.ndarray, target: np.ndarray, nbins: int = 64):
    """J = mean over non-empty bins of (S_b - target_b)^2 and its gradient dJ/dphi (full spectrum)."""
    S, cnt, _ = structure_factor(m, phi, nbins)
    sel = cnt > 0
    nb = int(sel.sum())
    J = float(np.sum((S[sel] - target[sel]) ** 2) / nb)
    coef = np.zeros(nbins)
    coef[sel] = 2.0 / nb * (S[sel] - target[sel]) * 2.0 / (m.n_sites * cnt[sel])
    return J, coef


def sq_bin_index(m: Model, nbins: int = 64) -> np.ndarray:
    """Bin of every full-spectrum mode (-1: not binned), same arithmetic as orc_structure_factor."""
    N = list(reversed(m.shape)) + [1] * (3 - m.dim)
    dx = list(m.dx) + [1.0] * 3
    ks = [np.fft.fftfreq(n) * n if n > 1 else np.zeros(1) for n in N]
    s2 = np.zeros((N[2], N[1], N[0]))
    for j, kk in enumerate((ks[0], ks[1], ks[2])):
        if N[j] == 1:
            continue
        t = (2.0 * nbins * kk * dx[0]) / (N[j] * dx[j])
        shape = [1, 1, 1]
        shape[2 - j] = N[j]
        s2 = s2 + (t * t).reshape(shape)
    s = np.sqrt(s2)
    b = np.ceil(s).astype(int) - 1
    b[(s2 == 0) | (s > nbins)] = -1
    return b.reshape(m.shape)

"""torch.autograd.Function over the GPU step and its hand-written adjoint.

``run(h0, params, system, param_ids, nsteps)`` advances a single-field system
``nsteps`` steps from the half spectrum ``h0`` with the named parameters set to
``params`` and returns the final half spectrum.  Its backward calls
``pss_adjoint_backward``: dJ/dh0 and dJ/dparams for the same noise
realisation (the step counter is reset to the run's first step, so that each
forward call draws the same noise).  Only marshalling happens here: the
library's gradient convention (dJ = Re sum over the full spectrum of
conj(lambda) dphi) is converted to PyTorch's (dJ = Re sum conj(grad) dh over
the stored half spectrum) by the Hermitian weights w = 1 on the kx = 0 and
kx = Nx/2 planes and 2 elsewhere.
"""
from __future__ import annotations

import numpy as np
import torch

from . import pss as _pss


def _weights(system: "_pss.System", device, dtype) -> torch.Tensor:
    w = torch.full((system.nx // 2 + 1,), 2.0, dtype=dtype, device=device)
    w[0] = 1.0
    w[-1] = 1.0
    return w


def _cdtype(system: "_pss.System"):
    return torch.complex128 if system.precision == "f64" else torch.complex64


class PSSRun(torch.autograd.Function):
    """The spectra stay on the device: h0, h_T, dJ/dh_T and dJ/dh0 are passed to the
    library as device pointers on PyTorch's current stream (the system is moved to
    that stream), so the run is ordered after the work that produced h0.  Only the
    parameter values (host doubles of the C ABI) cross to the host."""

    @staticmethod
    def forward(ctx, h0, params, system, param_ids, nsteps, step0):
        if not h0.is_cuda:
            raise ValueError("h0 must be a CUDA tensor (the half spectrum stays on the device)")
        sys_ = system
        sys_.set_stream(torch.cuda.current_stream(h0.device))
        for i, pid in enumerate(param_ids):
            sys_.set_param(pid, float(params[i]))
        sys_.set_step(step0)
        sys_.set_spectrum(0, h0.detach().to(_cdtype(sys_)).contiguous())
        sys_.adjoint_forward(int(nsteps))
        hT = torch.empty(sys_.half_shape, dtype=_cdtype(sys_), device=h0.device)
        sys_.get_spectrum(0, out=hT)
        ctx.system = sys_
        ctx.param_ids = list(param_ids)
        ctx.pdtype = params.dtype
        ctx.hdtype = h0.dtype
        return hT.to(h0.dtype)

    @staticmethod
    def backward(ctx, grad_hT):
        sys_ = ctx.system
        sys_.set_stream(torch.cuda.current_stream(grad_hT.device))
        rdt = torch.float64 if sys_.precision == "f64" else torch.float32
        w = _weights(sys_, grad_hT.device, rdt)
        lam_T = (grad_hT.detach().to(_cdtype(sys_)) / w).contiguous()
        n_all = len(sys_._param_names) if hasattr(sys_, "_param_names") else max(ctx.param_ids) + 1
        g_all, lam0 = sys_.adjoint_backward(lam_T, max(n_all, max(ctx.param_ids) + 1))
        g = torch.tensor([g_all[pid] for pid in ctx.param_ids], dtype=ctx.pdtype, device=grad_hT.device)
        grad_h0 = (lam0 * w).to(ctx.hdtype)
        return grad_h0, g, None, None, None, None


def run(h0: torch.Tensor, params: torch.Tensor, system: "_pss.System", param_ids, nsteps: int, step0: int = 0):
    """Differentiable ``nsteps``-step run of a single-field system (see module docstring)."""
    return PSSRun.apply(h0, params, system, tuple(param_ids), int(nsteps), int(step0))


def binned_structure_factor(h: torch.Tensor, shape, nbins: int = 64, dx: float = 1.0):
    """S(q) = |phi_q|^2 / N_sites averaged in nbins equal bins of 0 < |q| <= pi/dx (torch, differentiable);
    the bin of a mode is ceil(|q| nbins dx / pi) - 1.  Returns (S[nbins], counts[nbins])."""
    shape = tuple(shape)
    n = int(np.prod(shape))
    ks = [np.fft.fftfreq(m) * m for m in shape[:-1]] + [np.arange(shape[-1] // 2 + 1)]
    grids = np.meshgrid(*ks, indexing="ij")
    s2 = sum((2.0 * nbins * k / m) ** 2 for k, m in zip(grids, shape))
    s = np.sqrt(s2)
    b = np.ceil(s).astype(np.int64) - 1
    valid = (s2 > 0) & (s <= nbins)
    w = np.where(grids[-1] == 0, 1.0, 2.0)
    if shape[-1] % 2 == 0:
        w = np.where(grids[-1] == shape[-1] // 2, 1.0, w)
    w = np.where(valid, w, 0.0)
    bidx = torch.from_numpy(np.where(valid, b, 0).reshape(-1)).to(h.device)
    wt = torch.from_numpy(w.reshape(-1)).to(device=h.device, dtype=torch.float64)
    p = (h.reshape(-1).abs().to(torch.float64) ** 2) * wt / n
    sums = torch.zeros(nbins, dtype=torch.float64, device=h.device).index_add(0, bidx, p)
    cnt = torch.zeros(nbins, dtype=torch.float64, device=h.device).index_add(0, bidx, wt)
    return sums / cnt.clamp(min=1.0), cnt

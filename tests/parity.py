"""Comparison helpers of the GPU parity tests (numpy only; no step of the method).

A whole-array relative L2 norm is dominated by the largest (low-q) modes, so a
wrong Nyquist plane, a wrong last kept column or a wrong ragged last tile can
hide under it.  check_spectrum therefore also bounds every single mode:
max |got - ref| / rms(ref) over the whole half spectrum and, separately, over
the kx = 0 plane, the kx = Nx/2 plane, the last column the de-alias mask
keeps, and the last tile of 4 columns (ragged when Nx/2 + 1 is not a multiple
of 4: the device arrays hold the half spectrum in tiles of 4 columns).
"""
import numpy as np

TILE_W = 4          # columns per tile of the device layout
MODE_FACTOR = 10.0  # per-mode bound = MODE_FACTOR x the rel-L2 bar


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def kept_kx(nx, order):
    """Largest kx the per-axis mask keeps: (order + 1) kx < nx, at most nx / 2."""
    if order <= 0:
        return nx // 2
    k = (nx - 1) // (order + 1)
    return min(k, nx // 2)


def mode_errors(got, ref, order=2):
    """Per-region max |got - ref| / rms(ref) of half spectra [..., nx/2 + 1]."""
    got, ref = np.asarray(got), np.asarray(ref)
    assert got.shape == ref.shape, (got.shape, ref.shape)
    hx = ref.shape[-1]
    nx = 2 * (hx - 1)
    rms = max(float(np.sqrt(np.mean(np.abs(ref) ** 2))), 1e-300)
    d = np.abs(got - ref) / rms
    last_tile0 = ((hx - 1) // TILE_W) * TILE_W
    regions = {
        "all": d,
        "kx=0": d[..., 0],
        "kx=Nx/2": d[..., hx - 1],
        "last kept kx": d[..., kept_kx(nx, order)],
        "last tile": d[..., last_tile0:],
    }
    return {k: float(v.max()) for k, v in regions.items()}


def check_spectrum(got, ref, tol, order=2, what=""):
    """rel-L2 <= tol and every mode within MODE_FACTOR tol of rms(ref), per region.
    Returns (rel-L2, per-region maxima)."""
    err = rel(got, ref)
    modes = mode_errors(got, ref, order)
    bad = {k: v for k, v in modes.items() if not v <= MODE_FACTOR * tol}
    assert err <= tol and not bad, f"{what} rel-L2 {err:.3e} (bar {tol:g}); per-mode/rms {modes}"
    return err, modes


def check_real(got, ref, tol, what=""):
    """rel-L2 <= tol and every site within MODE_FACTOR tol of rms(ref)."""
    got, ref = np.asarray(got), np.asarray(ref)
    err = rel(got, ref)
    rms = max(float(np.sqrt(np.mean(np.abs(ref) ** 2))), 1e-300)
    worst = float(np.abs(got - ref).max() / rms)
    assert err <= tol and worst <= MODE_FACTOR * tol, f"{what} rel-L2 {err:.3e}, max/rms {worst:.3e} (bar {tol:g})"
    return err, worst

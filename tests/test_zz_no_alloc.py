"""pss_structure_factor_noalloc: the structure factor for callers that must not
allocate device memory while they run (their device memory is handed out up
front by another allocator, or they cannot afford cudaFree, which waits for
the whole device).  Its bin accumulator is a fixed array inside the library
that every call reuses, so each call must clear it first; the checks below
compare it with pss_structure_factor, which owns allocated scratch, on calls
made back to back.

This file is collected last on purpose, so that a run stopping at its first
failure has run every other test before this one.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-10, "f64": 1e-10}   # both sides sum the same values in FP64; only the order differs


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2405_02410_gb300 import build
    build.build()


def pss():
    from paper_2405_02410_gb300 import pss as m
    return m


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def same(got, want, tol):
    S, cnt, L = got
    S0, cnt0, L0 = want
    np.testing.assert_array_equal(cnt, cnt0)
    assert rel(S, S0) <= tol
    assert abs(L - L0) <= tol * abs(L0)


@pytest.mark.parametrize("shape,precision", [((128, 128), "f64"), ((32, 32, 32), "f32")])
def test_matches_allocating_entry_point_on_consecutive_calls(shape, precision):
    P = pss()
    s = P.model_b(shape, precision=precision, dt=0.01, a=-1, b=1, K=1, D=0.05, seed=7)
    s.init_uniform(0, -0.1, 0.1)
    s.step(20)
    tol = TOL[precision]
    # two calls in a row on the same state and bin count: a second call that
    # did not clear the array would report doubled sums
    first = s.structure_factor_noalloc(0, 64)
    second = s.structure_factor_noalloc(0, 64)
    want = s.structure_factor(0, 64)
    same(first, want, tol)
    same(second, want, tol)
    assert want[0].sum() > 0
    # a new state and a different bin count, then the largest bin count
    s.step(5)
    same(s.structure_factor_noalloc(0, 40), s.structure_factor(0, 40), tol)
    nmax = P.NOALLOC_MAX_BINS
    same(s.structure_factor_noalloc(0, nmax), s.structure_factor(0, nmax), tol)
    s.close()


def test_shared_array_across_systems():
    # two systems on one device share the array; calls made one after the
    # other (each synchronises) must not see each other's sums
    P = pss()
    a = P.model_b((64, 64), precision="f64", seed=1)
    b = P.model_b((128, 128), precision="f32", seed=2)
    a.init_uniform(0, -0.2, 0.2)
    b.init_uniform(0, -0.05, 0.05)
    a.step(3)
    b.step(3)
    for _ in range(2):
        same(a.structure_factor_noalloc(0, 32), a.structure_factor(0, 32), 1e-10)
        same(b.structure_factor_noalloc(0, 32), b.structure_factor(0, 32), 1e-10)
    a.close()
    b.close()


def test_rejects_more_bins_than_the_array_holds():
    P = pss()
    s = P.model_b((32, 32), precision="f64", seed=3)
    s.init_uniform(0, -0.1, 0.1)
    with pytest.raises(P.PssError) as err:
        s.structure_factor_noalloc(0, P.NOALLOC_MAX_BINS + 1)
    assert err.value.code == P.PSS_EINVAL
    assert str(P.NOALLOC_MAX_BINS) in str(err.value)
    with pytest.raises(P.PssError):
        s.structure_factor_noalloc(0, 0)
    # the handle stays usable after the rejected calls
    same(s.structure_factor_noalloc(0, 16), s.structure_factor(0, 16), 1e-10)
    s.close()

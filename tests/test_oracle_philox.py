"""Pins of the oracle's counter-based generator.

Philox4x32-10 is checked against an independent implementation: Triton's
``philox_impl`` executed by Triton's CPU interpreter (a library routine), on
random counters and keys.  The uniform and Box-Muller layers are checked by
their exact end points and by distribution statistics.
"""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from oracle import oracle as O
from tests import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_TRITON_SCRIPT = textwrap.dedent(
    """
    import os, sys
    os.environ["TRITON_INTERPRET"] = "1"
    import numpy as np, torch, triton, triton.language as tl

    @triton.jit
    def k(c0p, c1p, c2p, c3p, k0p, k1p, outp, N: tl.constexpr):
        i = tl.arange(0, N)
        u = lambda p: tl.load(p + i).to(tl.uint32, bitcast=True)
        a, b, c, d = tl.random.philox_impl(u(c0p), u(c1p), u(c2p), u(c3p), u(k0p), u(k1p), 10)
        tl.store(outp + i * 4 + 0, a.to(tl.int32, bitcast=True))
        tl.store(outp + i * 4 + 1, b.to(tl.int32, bitcast=True))
        tl.store(outp + i * 4 + 2, c.to(tl.int32, bitcast=True))
        tl.store(outp + i * 4 + 3, d.to(tl.int32, bitcast=True))

    data = np.load(sys.argv[1])
    ctr, key = data["ctr"], data["key"]
    N = ctr.shape[0]
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32))
    out = torch.zeros(4 * N, dtype=torch.int32)
    k[(1,)](t(ctr[:, 0]), t(ctr[:, 1]), t(ctr[:, 2]), t(ctr[:, 3]), t(key[:, 0]), t(key[:, 1]), out, N=N)
    np.save(sys.argv[2], out.numpy().view(np.uint32).reshape(N, 4))
    """
)


def test_philox_matches_triton_interpreter(tmp_path):
    pytest.importorskip("triton")
    n = 256
    ctr = inputs.uint32_counters(n, seed=21)
    key = inputs.uint32_keys(n, seed=22)
    ctr[0] = 0
    key[0] = 0
    ctr[1] = 0xFFFFFFFF
    key[1] = 0xFFFFFFFF
    np.savez(tmp_path / "in.npz", ctr=ctr, key=key)
    script = tmp_path / "t.py"
    script.write_text(_TRITON_SCRIPT)
    env = dict(os.environ, TRITON_INTERPRET="1")
    subprocess.run([sys.executable, str(script), str(tmp_path / "in.npz"), str(tmp_path / "out.npy")],
                   check=True, env=env, timeout=600, cwd=str(tmp_path))
    ref = np.load(tmp_path / "out.npy")
    got = np.stack([O.philox(ctr[i], key[i])[0] for i in range(n)])
    np.testing.assert_array_equal(got, ref)


def test_uniform24_end_points():
    assert O.uniform24(0) == 2.0 ** -25
    assert O.uniform24(0xFFFFFFFF) == 1.0 - 2.0 ** -25
    assert O.uniform24(0x80000000) == 0.5 + 2.0 ** -25
    # only the top 24 bits matter
    assert O.uniform24(0x123456FF) == O.uniform24(0x12345600)


def test_philox_uniform_statistics():
    n = 40000
    ctr = np.zeros((n, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(n)
    ctr[:, 1] = 7
    out = O.philox(ctr, np.array([2405, 0], dtype=np.uint32))
    u = np.array([O.uniform24(int(x)) for x in out[:, 0]])
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / n)
    assert abs(u.var() - 1 / 12) < 5 * np.sqrt(1 / 180 / n)
    hist, _ = np.histogram(u, bins=64, range=(0, 1))
    chi2 = np.sum((hist - n / 64) ** 2 / (n / 64))
    assert chi2 < 63 + 5 * np.sqrt(2 * 63)
    lag1 = np.corrcoef(u[:-1], u[1:])[0, 1]
    assert abs(lag1) < 5 / np.sqrt(n)
    # the four output words are not correlated with each other
    w = out.astype(np.float64)
    c = np.corrcoef(w.T)
    assert np.max(np.abs(c - np.eye(4))) < 5 / np.sqrt(n)


def test_box_muller_statistics():
    n = 20000
    z = np.array([O.normal_pair(99, i, 3, 1, 0) for i in range(n)])
    for col in range(2):
        v = z[:, col]
        assert abs(v.mean()) < 5 / np.sqrt(n)
        assert abs(v.var() - 1) < 5 * np.sqrt(2 / n)
        kurt = np.mean(v ** 4) / np.mean(v ** 2) ** 2
        assert abs(kurt - 3) < 0.15
    assert abs(np.corrcoef(z[:, 0], z[:, 1])[0, 1]) < 5 / np.sqrt(n)

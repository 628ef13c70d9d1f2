"""The paper's Model B example ("Example" section and its snapshot figure):
256 x 256, dt = 0.1, -a = b = 1, k = 4, no noise, a small random perturbation
of the uniform state, snapshots at t = 10, 100, 1000 and 5000.  Checked: the
first snapshot against the oracle, then what the section states (spinodal
decomposition into phi = +-1) and what it implies (exact mass conservation,
growing domains)."""
import math

import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2405_02410_gb300 import build
    build.build()


def test_spinodal_decomposition_of_the_example():
    from paper_2405_02410_gb300 import pss
    shape, dt = (256, 256), 0.1
    kw = dict(dt=dt, a=-1.0, b=1.0, K=4.0, D=0.0, noisy=False, seed=2405)
    s = pss.model_b(shape, precision="f32", **kw)
    s.init_uniform(0, -0.1, 0.1)
    mass0 = s.get_spectrum(0)[0, 0]
    L, t = {}, 0
    for T in (10, 100, 1000, 5000):
        s.step(int(round((T - t) / dt)))
        t = T
        L[T] = s.structure_factor(0, 64)[2]
        if T == 10:
            m = O.model_b(shape, **kw)
            ref = O.half(O.run(m, O.to_spectrum(m, O.init_uniform(m, -0.1, 0.1)), 0, 100))
            err = np.linalg.norm(s.get_spectrum(0) - ref) / np.linalg.norm(ref)
            assert err < 1e-4, err
    r = s.get_field(0)
    # two phases at phi = +-1 (the bulk of each domain), equal areas at zero mean
    assert abs(np.percentile(r, 97) - 1.0) < 0.05 and abs(np.percentile(r, 3) + 1.0) < 0.05
    assert 0.35 < np.mean(r > 0) < 0.65
    # the q = 0 mode is never touched by the update
    assert s.get_spectrum(0)[0, 0] == mass0
    # domains coarsen; between t = 1000 and 5000 the growth exponent is near the 1/3 of conserved dynamics
    assert L[10] < L[100] < L[1000] < L[5000]
    alpha = math.log(L[5000] / L[1000]) / math.log(5.0)
    assert 0.15 < alpha < 0.5, (alpha, L)

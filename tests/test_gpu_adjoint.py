"""The GPU adjoint (pss_adjoint_forward / pss_adjoint_backward) against the FP64
oracle adjoint and against finite differences of the GPU's own forward map."""
import numpy as np
import pytest

from oracle import oracle as O
from tests import inputs

from tests.parity import check_spectrum  # noqa: E402

pytestmark = pytest.mark.gpu


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
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


PARAMS = dict(a=-1.0, b=1.0, K=1.0, D=0.05)


def _weights(shape):
    k = np.meshgrid(*[np.fft.fftfreq(n) * n for n in shape], indexing="ij")
    kk = np.sqrt(sum(x ** 2 for x in k))
    return 1.0 + 0.5 * np.cos(0.4 * kk) ** 2


def _gpu_system(shape, prec, dt, seed, order=2):
    s = pss().model_b(shape, dt=dt, seed=seed, precision=prec, dealias_order=order, **PARAMS)
    s.init_uniform(0, -0.3, 0.3)
    return s


@pytest.mark.parametrize("shape,prec,tol", [
    ((32, 32), "f64", 1e-8), ((64,), "f64", 1e-8), ((8, 16, 8), "f64", 1e-8),
    ((32, 32), "f32", 1e-3), ((16, 16, 16), "f32", 1e-3),
])
def test_adjoint_matches_oracle(shape, prec, tol):
    dt, seed, n = 0.02, 17, 23
    m = O.model_b(shape, dt=dt, seed=seed, **PARAMS)
    phi0 = O.to_spectrum(m, O.init_uniform(m, -0.3, 0.3))
    c = _weights(shape)
    lamT = 2.0 * c * O.run(m, phi0, 0, n) / m.n_sites     # J = sum c |phi_T|^2 / N
    lam0, g = O.adjoint(m, phi0, 0, n, lamT)
    s = _gpu_system(shape, prec, dt, seed)
    s.adjoint_forward(n)
    grads, lam0_gpu = s.adjoint_backward(O.half(lamT), 4)
    assert rel(lam0_gpu, O.half(lam0)) < tol
    ref = np.array([g[1], -g[6], g[2], g[10]])             # (a, b, K, D) of Model B
    assert np.max(np.abs(grads - ref) / np.abs(ref)) < tol, (grads, ref)
    assert s.get_step() == n


def test_adjoint_structure_factor_loss_and_resume():
    # the binned S(q) loss of the adjoint workload, at 64 x 64
    shape, dt, seed, n, nb = (64, 64), 0.01, 2405, 40, 64
    m = O.model_b(shape, dt=dt, seed=seed, **PARAMS)
    phi0 = O.to_spectrum(m, O.init_uniform(m, -0.3, 0.3))
    phiT = O.run(m, phi0, 0, n)
    S, cnt, _ = O.structure_factor(m, phiT, nb)
    target = 0.9 * S
    J, coef = O.binned_sq_loss(m, phiT, target, nb)
    bins = O.sq_bin_index(m, nb)
    lamT = np.where(bins >= 0, coef[np.clip(bins, 0, None)], 0.0) * phiT
    lam0, g = O.adjoint(m, phi0, 0, n, lamT)
    s = _gpu_system(shape, "f64", dt, seed)
    s.adjoint_forward(n)
    grads, lam0_gpu = s.adjoint_backward(O.half(lamT), 4)
    assert rel(lam0_gpu, O.half(lam0)) < 1e-8
    np.testing.assert_allclose(grads, [g[1], -g[6], g[2], g[10]], rtol=1e-8)
    # the system is back at phi_T and keeps stepping from there
    check_spectrum(s.get_spectrum(0), O.half(phiT), 1e-12)
    s.step(5)
    check_spectrum(s.get_spectrum(0), O.half(O.run(m, phiT, n, 5)), 1e-12)


def test_adjoint_matches_gpu_finite_differences():
    shape, dt, seed, n = (32, 32), 0.02, 5, 15
    c = _weights(shape)
    w = np.ones(shape[-1] // 2 + 1) * 2.0
    w[0] = w[-1] = 1.0

    def J(**kw):
        p = dict(PARAMS)
        p.update(kw)
        s = pss().model_b(shape, dt=dt, seed=seed, precision="f64", **p)
        s.init_uniform(0, -0.3, 0.3)
        s.step(n)
        h = s.get_spectrum(0)
        return float(np.sum(w * O.half(c) * np.abs(h) ** 2) / (shape[0] * shape[1])), h

    J0, hT = J()
    s = _gpu_system(shape, "f64", dt, seed)
    s.adjoint_forward(n)
    grads, _ = s.adjoint_backward(2.0 * O.half(c) * hT / (shape[0] * shape[1]), 4)
    for i, name in enumerate(["a", "b", "K", "D"]):
        h = 1e-5
        fd = (J(**{name: PARAMS[name] + h})[0] - J(**{name: PARAMS[name] - h})[0]) / (2 * h)
        assert abs(grads[i] - fd) <= 1e-6 * abs(fd), (name, grads[i], fd)


def test_torch_autograd_function_matches_finite_differences():
    import torch
    from paper_2405_02410_gb300 import autograd as A
    shape, dt, n = (32, 32), 0.02, 12
    P = pss()
    s = P.model_b(shape, dt=dt, seed=9, precision="f64", **PARAMS)
    h0_np = np.fft.rfftn(inputs.real_field(shape, seed=3, lo=-0.3, hi=0.3))
    dev = torch.device("cuda")
    target = torch.linspace(0.01, 0.02, 16, dtype=torch.float64, device=dev)

    def loss(h0, params):
        hT = A.run(h0, params, s, [0, 1, 2, 3], n)
        S, cnt = A.binned_structure_factor(hT, shape, 16)
        sel = cnt > 0
        return ((S[sel] - target[sel]) ** 2).mean()

    h0 = torch.tensor(h0_np, device=dev, requires_grad=True)          # the spectra live on the device
    params = torch.tensor([PARAMS["a"], PARAMS["b"], PARAMS["K"], PARAMS["D"]], dtype=torch.float64,
                          device=dev, requires_grad=True)
    L = loss(h0, params)
    L.backward()
    # central differences in every parameter and along a random Hermitian direction of h0
    for i in range(4):
        e = torch.zeros(4, dtype=torch.float64, device=dev)
        e[i] = 1e-5
        fd = (loss(h0.detach(), params.detach() + e) - loss(h0.detach(), params.detach() - e)) / 2e-5
        assert abs(params.grad[i].item() - fd.item()) <= 1e-6 * abs(fd.item()), (i, params.grad[i], fd)
    d = torch.tensor(np.fft.rfftn(inputs.real_field(shape, seed=4)), device=dev)
    eps = 1e-4
    fd = (loss(h0.detach() + eps * d, params.detach()) - loss(h0.detach() - eps * d, params.detach())) / (2 * eps)
    ad = torch.real(torch.vdot(h0.grad.reshape(-1), d.reshape(-1)))
    assert abs(ad.item() - fd.item()) <= 1e-6 * abs(fd.item())


@pytest.mark.parametrize("shape", [(256, 256), (256, 512)])
def test_adjoint_on_the_fft_group_path(shape):
    # FP32 2D sides of 256..1024: the forward run and the backward pass's
    # recomputed steps take the FFT-group kernels (column-major product read
    # by the adjoint's column kernel); 13 steps = three segments of 4 and one
    # of 1, so the captured segment graph is replayed
    dt, seed, n = 0.02, 23, 13
    m = O.model_b(shape, dt=dt, seed=seed, **PARAMS)
    phi0 = O.to_spectrum(m, O.init_uniform(m, -0.3, 0.3))
    c = _weights(shape)
    lamT = 2.0 * c * O.run(m, phi0, 0, n) / m.n_sites
    lam0, g = O.adjoint(m, phi0, 0, n, lamT)
    ref = np.array([g[1], -g[6], g[2], g[10]])
    runs = {}
    for fast in (1, 0):
        s = _gpu_system(shape, "f32", dt, seed)
        s.set_tuning("fast2d", fast)
        assert s.step_path == (("persist2d" if shape[0] == shape[1] else "fast2d") if fast else "generic")
        s.adjoint_forward(n)
        grads, lam0_gpu = s.adjoint_backward(O.half(lamT), 4)
        assert rel(lam0_gpu, O.half(lam0)) < 1e-3
        assert np.max(np.abs(grads - ref) / np.abs(ref)) < 1e-3, (fast, grads, ref)
        assert s.get_step() == n
        runs[fast] = (grads, lam0_gpu)
    # the two paths agree to FP32 rounding
    assert rel(runs[1][1], runs[0][1]) < 1e-4
    assert np.max(np.abs(runs[1][0] - runs[0][0]) / np.abs(runs[0][0])) < 1e-4


@pytest.mark.parametrize("shape", [(256, 256), (512, 256), (256, 1024)])
def test_adjoint_x_pass_row_pairs_change_no_bit(shape):
    # the adjoint's x pass on FFT groups transforms each row pair on its own:
    # any number of pairs per CTA gives the same bits (automatic = spread over the SMs)
    dt, seed, n = 0.02, 31, 9
    m = O.model_b(shape, dt=dt, seed=seed, **PARAMS)
    lamT = 2.0 * _weights(shape) * O.run(m, O.to_spectrum(m, O.init_uniform(m, -0.3, 0.3)), 0, n) / m.n_sites
    out = {}
    for pairs in (0, 1, 2, 4, 8):
        s = _gpu_system(shape, "f32", dt, seed)
        assert s.step_path in ("fast2d", "persist2d")
        s.set_tuning("adj_row_pairs", pairs)
        s.adjoint_forward(n)
        out[pairs] = s.adjoint_backward(O.half(lamT), 4)
    for pairs in (1, 2, 4, 8):
        np.testing.assert_array_equal(out[pairs][1], out[0][1])
        np.testing.assert_allclose(out[pairs][0], out[0][0], rtol=1e-9)


@pytest.mark.parametrize("shape,prec", [((32, 32), "f64"), ((64,), "f64"), ((16, 16, 16), "f32"),
                                        ((8, 16, 8), "f64"), ((256, 256), "f32"), ((1024, 16), "f64")])
def test_fused_adjoint_launch_changes_no_field_bit(shape, prec):
    # part B of one adjoint step and part A of the step before it in one launch
    # (the default) or in two: the adjoint fields are the same bits, the FP64
    # gradient sums the same up to the order of their atomic additions; 11 steps
    # = segments of 4, 4 and 3
    dt, seed, n = 0.02, 29, 11
    m = O.model_b(shape, dt=dt, seed=seed, **PARAMS)
    lamT = 2.0 * _weights(shape) * O.run(m, O.to_spectrum(m, O.init_uniform(m, -0.3, 0.3)), 0, n) / m.n_sites
    out = {}
    for fuse in (1, 0):
        s = _gpu_system(shape, prec, dt, seed)
        s.set_tuning("persist_adj", 0)   # the per-step launches (the persistent pass has none to fuse)
        s.set_tuning("fuse_adjoint", fuse)
        s.adjoint_forward(n)
        l0 = s.launch_count
        grads, lam0 = s.adjoint_backward(O.half(lamT), 4)
        out[fuse] = (grads, lam0, s.launch_count - l0)
    np.testing.assert_array_equal(out[1][1], out[0][1])
    np.testing.assert_allclose(out[1][0], out[0][0], rtol=1e-12 if prec == "f64" else 1e-9)
    # the fused launch fits in shared memory everywhere but the FP64 1024-point column
    fits = not (prec == "f64" and shape[0] == 1024)
    if fits:
        assert out[1][2] < out[0][2], out
    else:
        assert out[1][2] == out[0][2], out


def test_adjoint_workload_recipe_at_64():
    # the adjoint workload's own recipe (Model B with the parity parameters, 64-bin
    # S(q) loss against the S(q) of a run with (a, b, K) = (-0.8, 1.2, 0.9) from the
    # same seed and initial field), at 64 x 64 and 200 steps: the FP32 GPU adjoint
    # against the FP64 oracle adjoint, the FP64 GPU adjoint against central
    # differences of the FP64 GPU forward run (h = 1e-4)
    shape, dt, seed, n, nb = (64, 64), 0.01, 2405, 200, 64
    base = dict(a=-1.0, b=1.0, K=1.0, D=0.01)
    m = O.model_b(shape, dt=dt, seed=seed, **base)
    phi0 = O.to_spectrum(m, O.init_uniform(m, -0.1, 0.1))
    mt = O.model_b(shape, dt=dt, seed=seed, a=-0.8, b=1.2, K=0.9, D=0.01)
    target, _, _ = O.structure_factor(mt, O.run(mt, phi0, 0, n), nb)
    bins = O.sq_bin_index(m, nb)

    def lam_of(phi_full, S, cnt):
        sel = cnt > 0
        coef = np.zeros(nb)
        coef[sel] = 2.0 / sel.sum() * (S[sel] - target[sel]) * 2.0 / (m.n_sites * cnt[sel])
        return np.where(bins >= 0, coef[np.clip(bins, 0, None)], 0.0) * phi_full

    # FP64 oracle adjoint
    phiT = O.run(m, phi0, 0, n)
    J, coef = O.binned_sq_loss(m, phiT, target, nb)
    lamT = np.where(bins >= 0, coef[np.clip(bins, 0, None)], 0.0) * phiT
    lam0, g = O.adjoint(m, phi0, 0, n, lamT)
    ref = np.array([g[1], -g[6], g[2], g[10]])

    def system(prec, **kw):
        p = dict(base)
        p.update(kw)
        s = pss().model_b(shape, dt=dt, seed=seed, precision=prec, **p)
        s.init_uniform(0, -0.1, 0.1)
        return s

    # FP32 GPU adjoint against the FP64 oracle adjoint
    s = system("f32")
    s.adjoint_forward(n)
    grads32, lam0_32 = s.adjoint_backward(O.half(lamT), 4)
    assert rel(lam0_32, O.half(lam0)) < 1e-3
    assert np.max(np.abs(grads32 - ref) / np.abs(ref)) < 1e-3, (grads32, ref)

    # FP64 GPU adjoint against FP64 GPU central differences of the same loss
    def J_gpu(**kw):
        s = system("f64", **kw)
        s.step(n)
        S, cnt, _ = s.structure_factor(0, nb)
        sel = cnt > 0
        return float(np.sum((S[sel] - target[sel]) ** 2) / sel.sum()), s

    J0, s64 = J_gpu()
    assert abs(J0 - J) <= 1e-10 * abs(J)
    S0, cnt0, _ = s64.structure_factor(0, nb)
    hT = s64.get_spectrum(0)
    full = np.fft.fftn(np.fft.irfftn(hT, s=shape, axes=(0, 1)))   # Hermitian completion (numpy)
    s = system("f64")
    s.adjoint_forward(n)
    grads64, _ = s.adjoint_backward(O.half(lam_of(full, S0, cnt0)), 4)
    # central differences at h = 1e-4 and h / 2, combined by Richardson extrapolation: the
    # noise amplitude is sqrt(D), whose third derivative at D = 0.01 leaves plain central
    # differences at h = 1e-4 about h^2 / (8 D^2) = 1.2e-5 off in dJ/dD
    h = 1e-4

    def central(name, step):
        return (J_gpu(**{name: base[name] + step})[0] - J_gpu(**{name: base[name] - step})[0]) / (2 * step)

    for i, name in enumerate(["a", "b", "K", "D"]):
        fd = (4.0 * central(name, h / 2) - central(name, h)) / 3.0
        assert abs(grads64[i] - fd) <= 1e-6 * abs(fd), (name, grads64[i], fd)
    np.testing.assert_allclose(grads64, ref, rtol=1e-8)


@pytest.mark.parametrize("shape", [(256, 256), (512, 256), (256, 1024)])
def test_adjoint_column_parts_on_fft_groups_match_the_generic_kernel(shape):
    # the column parts of the adjoint step (A, B and the fused B + A) on FFT groups,
    # one column per group, against the generic column kernel in its adjoint modes:
    # the same recursion, transforms of another radix layout, so FP32 rounding apart
    dt, seed, n = 0.02, 19, 11
    m = O.model_b(shape, dt=dt, seed=seed, **PARAMS)
    phi0 = O.to_spectrum(m, O.init_uniform(m, -0.3, 0.3))
    c = _weights(shape)
    lamT = 2.0 * c * O.run(m, phi0, 0, n) / m.n_sites
    lam0, g = O.adjoint(m, phi0, 0, n, lamT)
    ref = np.array([g[1], -g[6], g[2], g[10]])
    out = {}
    for groups in (1, 0):
        for fuse in (1, 0):
            s = _gpu_system(shape, "f32", dt, seed)
            s.set_tuning("persist_adj", 0)   # the column kernels themselves
            s.set_tuning("adj_col2", groups)
            s.set_tuning("fuse_adjoint", fuse)
            s.adjoint_forward(n)
            out[groups, fuse] = s.adjoint_backward(O.half(lamT), 4)
            grads, lam0_gpu = out[groups, fuse]
            assert rel(lam0_gpu, O.half(lam0)) < 1e-3
            assert np.max(np.abs(grads - ref) / np.abs(ref)) < 1e-3, (groups, fuse, grads, ref)
    # the fused and separate launches give the same adjoint field bits
    np.testing.assert_array_equal(out[1, 1][1], out[1, 0][1])
    np.testing.assert_allclose(out[1, 1][0], out[1, 0][0], rtol=1e-9)
    assert rel(out[1, 1][1], out[0, 1][1]) < 1e-4
    assert np.max(np.abs(out[1, 1][0] - out[0, 1][0]) / np.abs(out[0, 1][0])) < 1e-4


@pytest.mark.parametrize("shape,noisy", [((256, 256), True), ((512, 512), True), ((1024, 1024), True),
                                         ((256, 256), False)])
def test_persistent_backward_pass(shape, noisy):
    # each recomputed segment's backward pass as one persistent launch (the default on
    # the persistent path) against the per-step launches (column kernel on FFT groups,
    # fused B + A) and the FP64 oracle; 13 steps = segments of 4, 4, 4 and 1
    dt, seed, n = 0.02, 23, 13
    params = dict(PARAMS) if noisy else dict(PARAMS, D=0.0)
    m = O.model_b(shape, dt=dt, seed=seed, **params)
    phi0 = O.to_spectrum(m, O.init_uniform(m, -0.3, 0.3))
    c = _weights(shape)
    lamT = 2.0 * c * O.run(m, phi0, 0, n) / m.n_sites
    out = {}
    for persist_adj in (1, 0):
        s = pss().model_b(shape, dt=dt, seed=seed, precision="f32", **params)
        s.init_uniform(0, -0.3, 0.3)
        assert s.step_path == "persist2d"
        s.set_tuning("persist_adj", persist_adj)
        s.adjoint_forward(n)
        l0 = s.launch_count
        grads, lam0 = s.adjoint_backward(O.half(lamT), 4)
        out[persist_adj] = (grads, lam0, s.launch_count - l0)
        assert s.get_step() == n
    # the same recursion and transforms (the element-wise arithmetic may fuse
    # multiply-adds differently): FP32 rounding apart
    assert rel(out[1][1], out[0][1]) < 1e-5
    np.testing.assert_allclose(out[1][0], out[0][0], rtol=1e-5)
    assert out[1][2] < out[0][2], (out[1][2], out[0][2])
    if shape[0] <= 512:
        lam0, g = O.adjoint(m, phi0, 0, n, lamT)
        ref = np.array([g[1], -g[6], g[2], g[10]])
        assert rel(out[1][1], O.half(lam0)) < 1e-3
        k = 4 if noisy else 3
        assert np.max(np.abs(out[1][0][:k] - ref[:k]) / np.abs(ref[:k])) < 1e-3, (out[1][0], ref)


def test_adjoint_workload_at_its_own_size():
    # the adjoint workload itself: 2D Model B 256 x 256, 2000 steps (sqrt(n) = 45-step
    # segments), 64-bin S(q) loss against the S(q) of a run with (a, b, K) =
    # (-0.8, 1.2, 0.9) from the same seed and initial field.  The target comes from the
    # FP64 GPU run (the FP64 GPU path matches the oracle to 1e-10 in the parity tests;
    # a 2000-step oracle run at 256^2 takes about 30 s of one core).  The FP64 GPU
    # adjoint is checked against central differences of the FP64 GPU forward run with
    # Richardson extrapolation (h = 1e-4, h / 2) within 1e-6, the FP32 adjoint of the
    # persistent path against the FP64 adjoint within 1e-3 (measured: 4e-5)
    shape, dt, seed, n, nb = (256, 256), 0.01, 2405, 2000, 64
    base = dict(a=-1.0, b=1.0, K=1.0, D=0.01)

    def system(prec, **kw):
        p = dict(base)
        p.update(kw)
        s = pss().model_b(shape, dt=dt, seed=seed, precision=prec, **p)
        s.init_uniform(0, -0.1, 0.1)
        return s

    t = system("f64", a=-0.8, b=1.2, K=0.9)
    t.step(n)
    target, _, _ = t.structure_factor(0, nb)
    t.close()

    def loss(S, cnt):
        sel = cnt > 0
        return float(np.sum((S[sel] - target[sel]) ** 2) / sel.sum())

    def lam_T(s):
        # dJ/dphi_T on the half spectrum: (2 / nb)(S_b - S*_b) 2 / (N^2 cnt_b) phi_q in the bin of q
        h = s.get_spectrum(0)
        S, cnt, _ = s.structure_factor(0, nb)
        sel = cnt > 0
        coef = np.zeros(nb)
        coef[sel] = 2.0 / sel.sum() * (S[sel] - target[sel]) * 2.0 / (shape[0] * shape[1] * cnt[sel])
        ky = np.fft.fftfreq(shape[0]) * shape[0]
        kx = np.arange(shape[1] // 2 + 1)
        s2 = (2.0 * nb * ky[:, None] / shape[0]) ** 2 + (2.0 * nb * kx[None, :] / shape[1]) ** 2
        b = np.ceil(np.sqrt(s2)).astype(int) - 1
        ok = (s2 > 0) & (np.sqrt(s2) <= nb)
        return np.where(ok, coef[np.clip(b, 0, nb - 1)], 0.0) * h

    grads = {}
    for prec in ("f64", "f32"):
        s = system(prec)
        if prec == "f32":
            assert s.step_path == "persist2d"
        s.adjoint_forward(n)
        grads[prec], _ = s.adjoint_backward(lam_T(s).astype(np.complex128), 4)
        s.close()

    def J_gpu(**kw):
        s = system("f64", **kw)
        s.step(n)
        S, cnt, _ = s.structure_factor(0, nb)
        s.close()
        return loss(S, cnt)

    h = 1e-4

    def central(name, step):
        return (J_gpu(**{name: base[name] + step}) - J_gpu(**{name: base[name] - step})) / (2 * step)

    for i, name in enumerate(["a", "b", "K", "D"]):
        fd = (4.0 * central(name, h / 2) - central(name, h)) / 3.0
        assert abs(grads["f64"][i] - fd) <= 1e-6 * abs(fd), (name, grads["f64"][i], fd)
    assert np.max(np.abs(grads["f32"] - grads["f64"]) / np.abs(grads["f64"])) < 1e-3, (grads["f32"], grads["f64"])

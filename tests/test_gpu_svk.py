"""The spatially varying kernel on the GPU (the extension Sec. 1 cites, in the
Bramich et al. 2013 form: every kernel pixel a polynomial of degree dk in the
coordinates of Eq. 19) against the FP64 oracle's svk_* functions, which the
oracle tests pin by the pixel-by-pixel definition, central differences and
exact recovery of a drifting kernel.

Tolerances as for the constant kernel: loss and gradient <= 1e-5 relative
(max norm) at non-stationary theta; fitted kernels <= 1e-4 of sum K_00*,
background <= 1e-4 of the sky."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2104_13715_gb300 import synth
from tests._helpers import SPECS, ospec, rel_inf

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def nat():
    from paper_2104_13715_gb300 import native
    return native


def _nb(d):
    return (d + 1) * (d + 2) // 2


def varying_pair(H, W, m, seed, slope=(0.6, -0.4), shift=(0.5, 0.3), n_per_px=0.004):
    """A pair whose target PSF widens and drifts across the image."""
    spec = synth.PairSpec(size=(H, W), n_stars=max(3, int(n_per_px * H * W)), m=m, fwhm_ref=2.0,
                          kernel_sigma=1.0, scale=1.1, b0=25.0, sky=100.0, flux=(1e2, 1e5),
                          read=5.0, gain=1.0, kernel_sigma_slope=slope, shift_slope=shift)
    return synth.make_pair(spec, seed)


def theta_svk(m, dk, deg, I, rng, spread=0.3):
    """Box-car K_00 (jittered), small random coefficient kernels, B0 = median(I)
    and small higher background coefficients: a generic non-stationary point."""
    nk = m * m
    th = np.zeros(_nb(dk) * nk + _nb(deg))
    th[:nk] = 1.0 / nk * (1.0 + spread * rng.uniform(-1, 1, nk))
    th[nk:_nb(dk) * nk] = spread / nk * rng.uniform(-1, 1, (_nb(dk) - 1) * nk)
    th[_nb(dk) * nk] = float(np.median(I))
    th[_nb(dk) * nk + 1:] = rng.uniform(-5, 5, _nb(deg) - 1)
    return th


def _dev(a, dt=torch.float32):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)


@pytest.mark.parametrize("dk,m,name,deg", [(1, 3, "gauss-fixed", 0), (1, 7, "huber-ccd", 1),
                                           (1, 11, "cauchy-emccd", 0), (2, 5, "gauss-ccd", 2),
                                           (2, 9, "huber-fixed", 0), (1, 17, "gauss-fixed", 1),
                                           (2, 11, "gauss-emccd", 0)])
def test_loss_grad_matches_oracle(nat, dk, m, name, deg):
    spec = SPECS[name]
    d = varying_pair(150, 203, m, seed=10 * dk + m)
    rng = np.random.default_rng(m + dk)
    mask = (rng.random(d["R"].shape) > 0.08).astype(np.uint8)
    var = rng.uniform(50, 400, d["R"].shape).astype(np.float32) if spec["noise"] == "fixed" else None
    flat = rng.uniform(0.9, 1.1, d["R"].shape).astype(np.float32) if spec["noise"] != "fixed" else None
    th = theta_svk(m, dk, deg, d["I"], rng)
    L, g = nat.loss_grad(_dev(d["R"]), _dev(d["I"]), m, torch.from_numpy(th), nat.loss_spec(**spec),
                         mask=_dev(mask, torch.uint8), var=_dev(var), flat=_dev(flat),
                         bg_degree=deg, kernel_degree=dk)
    Lo, go = oracle.svk_loss_grad(d["R"], d["I"], m, th, dk, ospec(spec), mask=mask, var=var,
                                  flat=flat)
    assert L.item() == pytest.approx(Lo, rel=TOL)
    assert rel_inf(g.cpu().numpy(), go) <= TOL


def test_zero_coefficient_kernels_equal_the_constant_kernel(nat):
    """dk = 1 with K_01 = K_10 = 0 gives the constant-kernel loss and, for
    K_00 and the background, its gradient."""
    m, dk = 9, 1
    d = varying_pair(128, 160, m, seed=3)
    rng = np.random.default_rng(4)
    th = theta_svk(m, dk, 0, d["I"], rng)
    th[m * m:3 * m * m] = 0.0
    spec = nat.loss_spec(**SPECS["gauss-ccd"])
    R, I = _dev(d["R"]), _dev(d["I"])
    L1, g1 = nat.loss_grad(R, I, m, torch.from_numpy(th), spec, kernel_degree=dk)
    th0 = np.concatenate([th[:m * m], th[3 * m * m:]])
    L0, g0 = nat.loss_grad(R, I, m, torch.from_numpy(th0), spec)
    g1 = g1.cpu().numpy()
    assert L1.item() == pytest.approx(L0.item(), rel=TOL)
    assert rel_inf(np.concatenate([g1[:m * m], g1[3 * m * m:]]), g0.cpu().numpy()) <= TOL


def test_difference_image(nat):
    m, dk = 7, 2
    d = varying_pair(100, 140, m, seed=5)
    th = theta_svk(m, dk, 1, d["I"], np.random.default_rng(6))
    D = nat.diff_image(_dev(d["R"]), _dev(d["I"]), m, torch.from_numpy(th), bg_degree=1,
                       kernel_degree=dk).cpu().numpy()
    h = m // 2
    Do = d["I"][h:-h, h:-h] - oracle.svk_model(d["R"], th, m, dk)
    assert np.max(np.abs(D - Do)) <= 1e-5 * np.max(np.abs(d["I"]))


@pytest.mark.parametrize("dk", [1, 2])
def test_chi2_fit_matches_normal_equations(nat, dk):
    """dia_fit with the drifting-PSF target, fixed variance map: the
    spatially varying kernel's normal-equation solve of the oracle."""
    m = 9
    d = varying_pair(256, 272, m, seed=40 + dk)
    var = (25.0 + np.maximum(d["I"], 0.0)).astype(np.float32)
    spec = dict(rho="gauss", noise="fixed", var=1.0)
    out = nat.fit(_dev(d["R"]), _dev(d["I"]), m, nat.loss_spec(**spec), var=_dev(var),
                  kernel_degree=dk)
    assert out["info"]["status"] == 0, out["info"]
    th = out["theta"].cpu().numpy()
    ref = oracle.svk_normal_solve(d["R"], d["I"], m, dk, var=var)
    nk = m * m
    ek = np.max(np.abs(th[:-1] - ref[:-1])) / abs(ref[:nk].sum())
    eb = abs(th[-1] - ref[-1]) / float(np.median(d["I"]))
    assert ek <= 1e-4 and eb <= 1e-4, (ek, eb, out["info"])
    # the varying kernel fits better than one kernel (chi^2 of the residual)
    th1 = oracle.normal_solve(d["R"], d["I"], m, var=var)
    h = m // 2
    w = 1.0 / var[h:-h, h:-h]
    c_svk = np.sum(w * (d["I"][h:-h, h:-h] - oracle.svk_model(d["R"], ref, m, dk)) ** 2)
    c_one = np.sum(w * (d["I"][h:-h, h:-h] - oracle.model(d["R"], th1, m)) ** 2)
    assert c_svk < c_one


def test_ccd_fit_with_background_matches_newton(nat):
    """CCD negative log-likelihood, dk = 1, a degree-1 background: the FP64
    Newton optimum of the oracle polished from theta_gpu."""
    m, dk, deg = 7, 1, 1
    d = varying_pair(200, 208, m, seed=77)
    spec = SPECS["gauss-ccd"]
    out = nat.fit(_dev(d["R"]), _dev(d["I"]), m, nat.loss_spec(**spec), bg_degree=deg,
                  kernel_degree=dk)
    assert out["info"]["status"] == 0, out["info"]
    th = out["theta"].cpu().numpy()
    ref = oracle.svk_newton(d["R"], d["I"], m, th, dk, ospec(spec), max_iter=5)
    nk = m * m
    ek = np.max(np.abs(th[:3 * nk] - ref[:3 * nk])) / abs(ref[:nk].sum())
    sky = float(np.median(d["I"]))
    B = oracle.background_basis(d["R"].shape, m, deg)
    eb = np.max(np.abs(B @ (th[3 * nk:] - ref[3 * nk:]))) / sky
    assert ek <= 1e-4 and eb <= 1e-4, (ek, eb)


def test_fisher_matches_oracle_hessian(nat):
    m, dk = 5, 1
    d = varying_pair(120, 128, m, seed=9)
    th = theta_svk(m, dk, 0, d["I"], np.random.default_rng(2), spread=0.1)
    spec = SPECS["gauss-fixed"]
    var = (25.0 + np.maximum(d["I"], 0.0)).astype(np.float32)
    out = nat.fisher(_dev(d["R"]), _dev(d["I"]), m, torch.from_numpy(th), nat.loss_spec(**spec),
                     var=_dev(var), kernel_degree=dk)
    F = out["F"].cpu().numpy()
    Fo = oracle.svk_hessian(d["R"], d["I"], m, th, dk, ospec(spec), var=var)
    assert np.max(np.abs(F - Fo)) <= 1e-6 * np.max(np.abs(Fo))
    assert out["info"]["positive_definite"] == 1


def test_unsupported_uses_are_refused(nat):
    """Entries without a varying-kernel form refuse it; so does a theta
    larger than the optimiser holds and the regulariser (defined for one
    kernel); an out-of-range degree is an argument error."""
    R = torch.zeros((64, 64), device="cuda")
    spec = nat.loss_spec()
    p3, _ = nat.make_pair(R, R, 5, kernel_degree=1)
    th = torch.zeros(3 * 25 + 1, dtype=torch.float64, device="cuda")
    out = torch.zeros(3 * 25 + 2, dtype=torch.float64, device="cuda")
    vp = lambda t: ctypes.c_void_p(t.data_ptr())
    assert nat.lib.dia_loss_grad_noalloc(ctypes.byref(p3), ctypes.byref(spec), vp(th), vp(out),
                                         ctypes.c_void_p(out.data_ptr() + 8), None) == \
        nat.DIA_ERR_UNSUPPORTED
    D = torch.zeros((60, 60), device="cuda")
    ws = nat.pair_workspace(p3)
    assert nat.lib.dia_diff_image_tc(ctypes.byref(p3), vp(th), vp(D), vp(ws), ws.numel(),
                                     None) == nat.DIA_ERR_UNSUPPORTED
    pairs = (nat.Pair * 1)(p3)
    o = nat.default_opts()
    assert nat.lib.dia_fit_batch(pairs, 1, ctypes.byref(spec), ctypes.byref(o), None, None, None,
                                 None, 0, None) == nat.DIA_ERR_UNSUPPORTED
    big, _ = nat.make_pair(R, R, 15, kernel_degree=2)   # 6 x 225 + 1 > 1024
    ws2 = torch.zeros(1 << 20, dtype=torch.uint8, device="cuda")
    th2 = torch.zeros(6 * 225 + 1, dtype=torch.float64, device="cuda")
    assert nat.lib.dia_loss_grad(ctypes.byref(big), ctypes.byref(spec), vp(th2), vp(out), vp(out),
                                 vp(ws2), ws2.numel(), None) == nat.DIA_ERR_UNSUPPORTED
    reg = nat.default_opts(reg_lambda=1.0)
    assert nat.lib.dia_fit(ctypes.byref(p3), ctypes.byref(spec), ctypes.byref(reg), None, None,
                           None, None, None, None, vp(ws), ws.numel(), None) == \
        nat.DIA_ERR_UNSUPPORTED
    bad, _ = nat.make_pair(R, R, 5, kernel_degree=3)
    assert nat.lib.dia_pair_workspace_size(ctypes.byref(bad), 0) == 0

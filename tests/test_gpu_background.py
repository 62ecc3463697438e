"""Polynomial spatial background (Sec. 2.6, Eq. 18-19) through the C ABI against
the FP64 oracle.

Tolerances: gradients <= 1e-5 relative in the max norm and the loss <= 1e-5
relative at non-stationary theta (as for the constant background); fitted
kernels max |K - K*| <= 1e-4 |sum K*|; fitted backgrounds max |B - B*| over
the valid region <= 1e-4 x sky (the constant-background bound on B0, applied
to the whole background surface); difference images to 1e-6 of max |I|."""
import numpy as np
import pytest
import torch

import oracle
from tests._helpers import SPECS, field, ospec, rel_inf, theta_start

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nat():
    from paper_2104_13715_gb300 import native
    return native


def _t(a, dt=torch.float32):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)


def _coef(deg, rng, sky):
    """Background coefficients b_00 ... b_d0 of a smooth surface around sky."""
    c = rng.uniform(-0.3, 0.3, oracle.n_background(deg)) * sky
    c[0] = sky
    return c


def _with_background(d, m, deg, seed, sky=100.0):
    """The pair of `field` with a degree-d polynomial (Eq. 18, on the full
    image grid) added to the target; returns (pair dict, coefficients)."""
    rng = np.random.default_rng(seed)
    H, W = d["I"].shape
    c = _coef(deg, rng, sky)
    y, x = np.mgrid[0:H, 0:W].astype(float)
    eta, xi = (x - (W - 1) / 2) / W, (y - (H - 1) / 2) / H
    B = np.zeros((H, W))
    k = 0
    for p in range(deg + 1):
        for q in range(deg - p + 1):
            B += c[k] * eta ** p * xi ** q
            k += 1
    out = dict(d)
    out["I"] = (d["I"] + B - sky).astype(np.float32)
    return out, c


def _bg_err(theta, ref, shape, m, deg):
    """max |B(theta) - B(ref)| over the valid region."""
    Bs = oracle.background_basis(shape, m, deg)
    nk = m * m
    return float(np.max(np.abs(Bs @ (theta[nk:] - ref[nk:]))))


def _check_fit(theta, ref, shape, m, deg, sky, tol=1e-4):
    nk = m * m
    ek = np.max(np.abs(theta[:nk] - ref[:nk])) / abs(ref[:nk].sum())
    eb = _bg_err(theta, ref, shape, m, deg) / sky
    assert ek <= tol and eb <= tol, (ek, eb)


@pytest.mark.parametrize("deg", [1, 2, 3, 4])
@pytest.mark.parametrize("name", ["gauss-fixed", "gauss-ccd", "cauchy-emccd"])
def test_loss_grad_with_polynomial_background(nat, deg, name):
    m = 9
    d0 = field(170, 300, m, seed=50 + deg)
    d, c = _with_background(d0, m, deg, seed=deg)
    spec = SPECS[name]
    rng = np.random.default_rng(deg)
    th = np.concatenate([theta_start(m, d["I"], rng, 0.3)[:-1], c * (1 + 0.05 * rng.normal(size=c.size))])
    mask = (rng.random(d["I"].shape) > 0.03).astype(np.uint8)
    Lo, go = oracle.loss_grad(d["R"], d["I"], m, th, ospec(spec), mask=mask)
    for fn in (nat.loss_grad, nat.loss_grad_noalloc):
        L, g = fn(_t(d["R"]), _t(d["I"]), m, torch.from_numpy(th), nat.loss_spec(**spec),
                  mask=_t(mask, torch.uint8), bg_degree=deg)
        assert g.numel() == m * m + oracle.n_background(deg)
        assert rel_inf(g.cpu().numpy(), go) <= 1e-5
        assert abs(L.item() - Lo) <= 1e-5 * abs(Lo)


def test_degree_zero_is_the_constant_background(nat):
    """bg_degree 0 and a degree-2 theta with zero higher coefficients give the
    same loss and the same kernel/B0 gradient."""
    m = 7
    d = field(130, 140, m, seed=60)
    spec = nat.loss_spec(**SPECS["gauss-ccd"])
    th0 = theta_start(m, d["I"], np.random.default_rng(60), 0.2)
    th2 = np.concatenate([th0, np.zeros(5)])
    L0, g0 = nat.loss_grad(_t(d["R"]), _t(d["I"]), m, torch.from_numpy(th0), spec)
    L2, g2 = nat.loss_grad(_t(d["R"]), _t(d["I"]), m, torch.from_numpy(th2), spec, bg_degree=2)
    assert abs(L0.item() - L2.item()) <= 1e-6 * abs(L0.item())
    assert rel_inf(g2.cpu().numpy()[: m * m + 1], g0.cpu().numpy()) <= 1e-6


def test_diff_image_with_polynomial_background(nat):
    m, deg = 11, 3
    d, c = _with_background(field(200, 190, m, seed=61), m, deg, seed=61)
    th = np.concatenate([oracle.normal_solve(d["R"], d["I"], m)[:-1], c])
    D = nat.diff_image(_t(d["R"]), _t(d["I"]), m, torch.from_numpy(th), bg_degree=deg)
    Do = oracle.diff_image(d["R"], d["I"], m, th)
    assert np.max(np.abs(D.cpu().numpy() - Do)) <= 1e-6 * np.max(np.abs(d["I"]))


@pytest.mark.parametrize("deg", [1, 2, 4])
@pytest.mark.parametrize("precond,adam", [(1, 5000), (1, 0), (0, 0)])
def test_chi2_fit_recovers_the_normal_solution(nat, deg, precond, adam):
    m, sky = 11, 100.0
    d, _ = _with_background(field(256, 240, m, seed=70 + deg), m, deg, seed=70 + deg, sky=sky)
    ref = oracle.normal_solve(d["R"], d["I"], m, deg=deg)
    out = nat.fit(_t(d["R"]), _t(d["I"]), m, nat.loss_spec(**SPECS["gauss-fixed"]),
                  nat.default_opts(precond=precond, max_adam_iters=adam,
                                   history=20 if precond else 100),
                  bg_degree=deg)
    th = out["theta"].cpu().numpy()
    assert out["info"]["status"] == 0, out["info"]
    assert th.size == m * m + oracle.n_background(deg)
    _check_fit(th, ref, d["I"].shape, m, deg, sky)
    assert out["b0"].item() == pytest.approx(th[m * m], rel=1e-6)
    D = out["diff"].cpu().numpy()
    assert np.max(np.abs(D - oracle.diff_image(d["R"], d["I"], m, th))) <= 1e-6 * np.max(np.abs(d["I"]))


@pytest.mark.parametrize("name", ["gauss-ccd", "huber-ccd"])
def test_likelihood_fit_is_the_newton_optimum(nat, name):
    m, deg, sky = 9, 2, 150.0
    d, _ = _with_background(field(180, 200, m, seed=80, sky=sky), m, deg, seed=80, sky=sky)
    spec = SPECS[name]
    out = nat.fit(_t(d["R"]), _t(d["I"]), m, nat.loss_spec(**spec),
                  nat.default_opts(max_adam_iters=0), bg_degree=deg)
    th = out["theta"].cpu().numpy()
    assert out["info"]["status"] == 0
    ref = oracle.newton(d["R"], d["I"], m, th, ospec(spec))
    _check_fit(th, ref, d["I"].shape, m, deg, sky)


def test_background_with_regulariser_and_clipping(nat):
    """Degree 1 with the kernel regulariser (Eq. 20) and two sigma-clip refits:
    the final theta is the regularised normal solution on the final mask."""
    m, deg, lam, sky = 9, 1, 2.0, 100.0
    d, _ = _with_background(field(200, 210, m, seed=90), m, deg, seed=90, sky=sky)
    d["I"][40, 50] += 5000.0
    d["I"][120, 100] -= 3000.0
    var = (25.0 + np.maximum(d["I"], 0)).astype(np.float32)   # read noise 5 + Poisson
    out = nat.fit(_t(d["R"]), _t(d["I"]), m, nat.loss_spec(**SPECS["gauss-fixed"]),
                  nat.default_opts(reg_lambda=lam, clip_passes=2), var=_t(var), want_mask=True,
                  bg_degree=deg)
    th = out["theta"].cpu().numpy()
    mk = out["mask"].cpu().numpy()
    assert out["info"]["status"] == 0
    assert mk[40, 50] == 0 and mk[120, 100] == 0
    assert mk.mean() > 0.95
    ref = oracle.normal_solve(d["R"], d["I"], m, mask=mk, var=var, reg_lambda=lam, deg=deg)
    _check_fit(th, ref, d["I"].shape, m, deg, sky)


@pytest.mark.parametrize("precond", [1, 0])
def test_batch_with_mixed_degrees(nat, precond):
    sky = 100.0
    cases = [(5, 0), (9, 2), (13, 1), (7, 4), (11, 3)]
    ds = []
    for i, (m, deg) in enumerate(cases):
        d, _ = _with_background(field(96 + 24 * i, 110 + 8 * i, m, seed=100 + i), m, deg,
                                seed=100 + i, sky=sky)
        ds.append(d)
    items = [dict(R=_t(d["R"]), I=_t(d["I"]), m=m, bg_degree=deg) for d, (m, deg) in zip(ds, cases)]
    out = nat.fit_batch(items, nat.loss_spec(**SPECS["gauss-fixed"]),
                        nat.default_opts(precond=precond, history=20 if precond else 100))
    assert out["status"] == 0
    for d, (m, deg), th, info in zip(ds, cases, out["thetas"], out["infos"]):
        assert info["status"] == 0
        ref = oracle.normal_solve(d["R"], d["I"], m, deg=deg)
        _check_fit(th.cpu().numpy(), ref, d["I"].shape, m, deg, sky)


def test_fisher_with_polynomial_background(nat):
    """F of the fixed-variance chi^2 with a degree-2 background: element-wise
    within 1e-6 of max |F| of the oracle's Hessian, covariance its inverse."""
    m, deg = 7, 2
    d, c = _with_background(field(120, 130, m, seed=110), m, deg, seed=110)
    th = oracle.normal_solve(d["R"], d["I"], m, deg=deg)
    spec = SPECS["gauss-fixed"]
    out = nat.fisher(_t(d["R"]), _t(d["I"]), m, _t(th, torch.float64), nat.loss_spec(**spec),
                     bg_degree=deg)
    F = out["F"].cpu().numpy()
    H = oracle.hessian(d["R"], d["I"], m, th, ospec(spec))
    assert F.shape == H.shape == (m * m + 6, m * m + 6)
    assert np.max(np.abs(F - H)) <= 1e-6 * np.max(np.abs(H))
    assert out["info"]["positive_definite"] == 1 and out["info"]["n"] == m * m + 6
    cov = out["cov"].cpu().numpy()
    ref_inv = np.linalg.inv(F)
    assert np.max(np.abs(cov - ref_inv)) <= 1e-7 * np.max(np.abs(ref_inv))


def test_host_buffers_and_theta0_with_background(nat):
    """Host (pinned) buffers staged by the library give the device result
    bitwise; a fit started from theta0 (init 2) of the background length
    lands on the same optimum."""
    m, deg, sky = 7, 2, 100.0
    d, c = _with_background(field(140, 150, m, seed=120), m, deg, seed=120, sky=sky)
    spec = nat.loss_spec(**SPECS["gauss-fixed"])
    R = torch.from_numpy(d["R"]).pin_memory()
    I = torch.from_numpy(d["I"]).pin_memory()
    host = nat.fit(R, I, m, spec, bg_degree=deg)
    assert not host["theta"].is_cuda and host["theta"].numel() == m * m + 6
    dev = nat.fit(_t(d["R"]), _t(d["I"]), m, spec, bg_degree=deg)
    assert np.array_equal(dev["theta"].cpu().numpy(), host["theta"].numpy())
    ref = oracle.normal_solve(d["R"], d["I"], m, deg=deg)
    _check_fit(host["theta"].numpy(), ref, d["I"].shape, m, deg, sky)
    th0 = np.concatenate([np.full(m * m, 1.0 / (m * m)), c])
    warm = nat.fit(_t(d["R"]), _t(d["I"]), m, spec, theta0=th0, bg_degree=deg)
    _check_fit(warm["theta"].cpu().numpy(), ref, d["I"].shape, m, deg, sky)
    with pytest.raises(ValueError):
        nat.fit(_t(d["R"]), _t(d["I"]), m, spec, theta0=th0[:-1], bg_degree=deg)

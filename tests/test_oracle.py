"""Pins of the FP64 oracle against things other than itself: library routines
(scipy correlate / log-densities / Huber, numpy lstsq), closed forms, finite
differences, the paper's invariants (Sec. 3.4) and its printed values."""
import json
import math
import os

import numpy as np
import pytest
from scipy import signal, special, stats

import oracle
from oracle import LossSpec

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _star_ref(shape, n, sigma, rng, flux=(50, 5000)):
    """A small smooth star-field-like reference, built in the test."""
    H, W = shape
    yy, xx = np.mgrid[0:H, 0:W]
    img = np.zeros(shape)
    for _ in range(n):
        x0, y0 = rng.uniform(0, W), rng.uniform(0, H)
        f = rng.uniform(*flux)
        img += f * np.exp(-((xx - x0) ** 2 + (yy - y0) ** 2) / (2 * sigma * sigma))
    return img + rng.normal(0, 1.0, shape)


def _scipy_model(R, theta, m):
    K = theta[:-1].reshape(m, m)
    return signal.correlate2d(R, K, mode="valid") + theta[-1]


def _valid(a, m):
    h = m // 2
    return a[h:a.shape[0] - h, h:a.shape[1] - h]


# ---------------------------------------------------------------- model image
@pytest.mark.parametrize("shape,m", [((13, 17), 5), ((9, 9), 9), ((6, 11), 1), ((20, 7), 3)])
def test_model_matches_scipy_correlate(shape, m):
    rng = np.random.default_rng(1)
    R = rng.normal(size=shape)
    th = rng.normal(size=m * m + 1)
    np.testing.assert_allclose(oracle.model(R, th, m), _scipy_model(R, th, m),
                               rtol=0, atol=1e-12)


def test_ndata_golden():
    g = GOLD["ndata_142_m19"]["value"]
    assert oracle.ndata((142, 142), 19) == g
    mask = np.ones((142, 142), np.uint8)
    mask[50, 60] = 0          # inside the valid region
    mask[0, 0] = 0            # outside: does not count anyway
    assert oracle.ndata((142, 142), 19, mask) == g - 1


# ------------------------------------------------------------------ the loss
def _case(seed=0, shape=(12, 14), m=3):
    rng = np.random.default_rng(seed)
    R = rng.uniform(0, 50, shape)
    th = np.concatenate([rng.uniform(0.05, 0.15, m * m), [20.0]])
    I = _scipy_model(R, th, m)
    h = m // 2
    I_full = np.zeros(shape)
    I_full[h:shape[0] - h, h:shape[1] - h] = I + rng.normal(0, 3.0, I.shape)
    I_full[I_full == 0] = 1.0
    th0 = th + rng.normal(0, 0.02, th.shape)
    return R, I_full, th0


def test_gauss_fixed_loss_is_gaussian_nll_minus_constants():
    R, I, th = _case()
    m = 3
    rng = np.random.default_rng(5)
    var = rng.uniform(1.0, 9.0, I.shape)
    mask = (rng.random(I.shape) > 0.2).astype(np.uint8)
    L, _ = oracle.loss_grad(R, I, m, th, LossSpec("gauss", "fixed"), mask=mask, var=var)
    M = _scipy_model(R, th, m)
    w = _valid(mask, m) != 0
    sd = np.sqrt(_valid(var, m))
    nll = -stats.norm.logpdf(_valid(I, m), loc=M, scale=sd)
    # Eq. 4 minus the sigma-only constants: 1/2 chi^2 over the unmasked pixels
    ref = np.sum((nll - np.log(sd) - 0.5 * math.log(2 * math.pi))[w])
    assert L == pytest.approx(ref, rel=1e-12)


@pytest.mark.parametrize("noise", ["ccd", "emccd"])
def test_model_dependent_nll_is_gaussian_logpdf(noise):
    R, I, th = _case(2)
    m = 3
    rng = np.random.default_rng(7)
    flat = rng.uniform(0.8, 1.2, I.shape)
    spec = LossSpec("gauss", noise, sigma0=4.0, gain=1.7, excess=2.0)
    L, _ = oracle.loss_grad(R, I, m, th, spec, flat=flat)
    M = _scipy_model(R, th, m)
    F = _valid(flat, m)
    if noise == "ccd":
        v = 16.0 / F ** 2 + M / (1.7 * F)          # Eq. 6
    else:
        v = 2.0 * M / (1.7 * F)                     # Eq. 7
    ref = -np.sum(stats.norm.logpdf(_valid(I, m), loc=M, scale=np.sqrt(v)))
    ref -= M.size * 0.5 * math.log(2 * math.pi)
    assert L == pytest.approx(ref, rel=1e-12)


def test_huber_loss_matches_scipy_huber():
    R, I, th = _case(3)
    m = 3
    c = GOLD["huber_c"]["value"]
    spec = LossSpec("huber", "ccd", sigma0=3.0, gain=2.0, huber_c=c)
    L, _ = oracle.loss_grad(R, I, m, th, spec)
    M = _scipy_model(R, th, m)
    v = 9.0 + M / 2.0
    z = (_valid(I, m) - M) / np.sqrt(v)
    assert np.any(np.abs(z) > c) and np.any(np.abs(z) < c)
    ref = np.sum(special.huber(c, z)) + np.sum(0.5 * np.log(v))   # Eq. 13 without Q
    assert L == pytest.approx(ref, rel=1e-12)


def test_cauchy_loss_matches_scipy_cauchy():
    R, I, th = _case(4)
    m = 3
    var = np.full(I.shape, 4.0)
    L, _ = oracle.loss_grad(R, I, m, th, LossSpec("cauchy", "fixed"), var=var)
    M = _scipy_model(R, th, m)
    z = (_valid(I, m) - M) / 2.0
    ref = np.sum(-stats.cauchy.logpdf(z) - math.log(math.pi))
    assert L == pytest.approx(ref, rel=1e-12)


def test_huber_large_c_is_gaussian():
    R, I, th = _case(5)
    a = oracle.loss_grad(R, I, 3, th, LossSpec("huber", "ccd", sigma0=3, gain=2, huber_c=1e9))
    b = oracle.loss_grad(R, I, 3, th, LossSpec("gauss", "ccd", sigma0=3, gain=2))
    assert a[0] == pytest.approx(b[0], rel=1e-14)
    np.testing.assert_allclose(a[1], b[1], rtol=1e-13)


def test_variance_floor_clamps():
    # EMCCD with a negative model value: v is clamped at the floor
    R = np.zeros((5, 5))
    I = np.full((5, 5), 3.0)
    th = np.zeros(10)
    th[-1] = -1.0                          # M = -1 everywhere
    spec = LossSpec("gauss", "emccd", gain=1.0, excess=2.0, var_floor=0.5)
    L, g = oracle.loss_grad(R, I, 3, th, spec)
    n = 9
    assert L == pytest.approx(n * (0.5 * 16 / 0.5 + 0.5 * math.log(0.5)), rel=1e-14)
    # dv/dM = 0 where clamped: dl/dM = -(I - M)/v
    assert g[-1] == pytest.approx(n * (-4.0 / 0.5), rel=1e-14)


ALL_SPECS = [
    LossSpec("gauss", "fixed"),
    LossSpec("gauss", "ccd", sigma0=4.0, gain=1.5),
    LossSpec("gauss", "emccd", gain=0.086, excess=2.0),
    LossSpec("huber", "fixed", huber_c=1.345),
    LossSpec("huber", "ccd", sigma0=2.0, gain=1.5, huber_c=1.345),
    LossSpec("cauchy", "fixed"),
    LossSpec("cauchy", "emccd", gain=0.5, excess=2.0),
]


@pytest.mark.parametrize("spec", ALL_SPECS, ids=lambda s: f"{s.rho}-{s.noise}")
def test_gradient_central_differences(spec):
    R, I, th = _case(6, shape=(9, 10), m=3)
    rng = np.random.default_rng(11)
    var = rng.uniform(1, 5, I.shape)
    flat = rng.uniform(0.9, 1.1, I.shape)
    mask = np.ones(I.shape, np.uint8)
    mask[4, 5] = 0
    kw = dict(mask=mask, var=var if spec.noise == "fixed" else None,
              flat=flat if spec.noise != "fixed" else None)
    L, g = oracle.loss_grad(R, I, 3, th, spec, **kw)
    for k in range(th.size):
        e = 1e-6 * max(1.0, abs(th[k]))
        tp, tm = th.copy(), th.copy()
        tp[k] += e
        tm[k] -= e
        fd = (oracle.loss(R, I, 3, tp, spec, **kw) - oracle.loss(R, I, 3, tm, spec, **kw)) / (2 * e)
        assert fd == pytest.approx(g[k], rel=2e-6, abs=1e-6 * np.max(np.abs(g)))


@pytest.mark.parametrize("spec", ALL_SPECS, ids=lambda s: f"{s.rho}-{s.noise}")
def test_hessian_central_differences(spec):
    R, I, th = _case(8, shape=(8, 9), m=3)
    Hm = oracle.hessian(R, I, 3, th, spec)
    for k in range(th.size):
        e = 1e-5 * max(1.0, abs(th[k]))
        tp, tm = th.copy(), th.copy()
        tp[k] += e
        tm[k] -= e
        fd = (oracle.loss_grad(R, I, 3, tp, spec)[1] - oracle.loss_grad(R, I, 3, tm, spec)[1]) / (2 * e)
        np.testing.assert_allclose(Hm[:, k], fd, rtol=1e-5, atol=1e-6 * np.max(np.abs(Hm)))


# ------------------------------------------------------- normal equations (B08)
def test_normal_solve_matches_lstsq_on_explicit_design_matrix():
    rng = np.random.default_rng(3)
    shape, m = (21, 19), 5
    R = _star_ref(shape, 6, 1.3, rng)
    I = rng.normal(0, 2.0, shape) + 10.0
    I += 0.9 * np.roll(np.roll(R, 1, 0), -1, 1)
    var = rng.uniform(1.0, 4.0, shape)
    h = m // 2
    rows, rhs = [], []
    for i in range(h, shape[0] - h):          # explicit design matrix, one row per pixel
        for j in range(h, shape[1] - h):
            phi = [R[i - h + a, j - h + b] for a in range(m) for b in range(m)] + [1.0]
            w = 1.0 / math.sqrt(var[i, j])
            rows.append([w * p for p in phi])
            rhs.append(w * I[i, j])
    ref = np.linalg.lstsq(np.array(rows), np.array(rhs), rcond=None)[0]
    th = oracle.normal_solve(R, I, m, var=var)
    np.testing.assert_allclose(th, ref, rtol=1e-8, atol=1e-9 * np.max(np.abs(ref)))


def test_normal_solve_is_the_chi2_minimum():
    rng = np.random.default_rng(4)
    R = _star_ref((24, 24), 8, 1.5, rng)
    I = 1.1 * R + 5 + rng.normal(0, 1, R.shape)
    th = oracle.normal_solve(R, I, 5)
    _, g = oracle.loss_grad(R, I, 5, th, LossSpec())
    _, g0 = oracle.loss_grad(R, I, 5, np.zeros_like(th), LossSpec())
    assert np.max(np.abs(g)) < 1e-9 * np.max(np.abs(g0))


def test_identical_images_give_delta_kernel():
    """Sec. 3.4 test (i)."""
    rng = np.random.default_rng(0)
    R = _star_ref((30, 30), 12, 1.4, rng)
    m = 7
    th = oracle.normal_solve(R, R.copy(), m)
    K = th[:-1].reshape(m, m)
    d = np.zeros((m, m))
    d[m // 2, m // 2] = 1.0
    np.testing.assert_allclose(K, d, atol=1e-9)
    assert abs(th[-1]) < 1e-8


def test_plus_one_pixel_shift_gives_delta_at_minus_one():
    """Sec. 3.4 test (iii): the orientation of the kernel offsets."""
    rng = np.random.default_rng(1)
    R = _star_ref((32, 32), 12, 1.4, rng)
    I = np.zeros_like(R)
    I[1:, 1:] = R[:-1, :-1]                    # target moved by +1 in x and y
    m = 5
    th = oracle.normal_solve(R, I, m)
    K = th[:-1].reshape(m, m)
    dl, dm = GOLD["shift_plus1_delta_offset"]["value"]
    peak = np.unravel_index(np.argmax(K), K.shape)
    assert (peak[0] - m // 2, peak[1] - m // 2) == (dl, dm)
    d = np.zeros((m, m))
    d[m // 2 + dl, m // 2 + dm] = 1.0
    np.testing.assert_allclose(K, d, atol=1e-9)


def test_noiseless_gaussian_kernel_recovered():
    """Sec. 3.4 test (ii): a Gaussian kernel phi_K = 1.5 with a scale and a
    background is recovered exactly by the FP64 normal equations."""
    rng = np.random.default_rng(2)
    R = _star_ref((48, 48), 25, 1.2, rng)
    m = 9
    yy, xx = np.mgrid[-4:5, -4:5]
    Kt = np.exp(-(xx ** 2 + yy ** 2) / (2 * 1.5 ** 2))
    Kt *= 1.3 / Kt.sum()
    I = np.zeros_like(R)
    I[4:-4, 4:-4] = signal.correlate2d(R, Kt, mode="valid") + 17.0
    th = oracle.normal_solve(R, I, m)
    np.testing.assert_allclose(th[:-1].reshape(m, m), Kt, atol=1e-9)
    assert th[-1] == pytest.approx(17.0, abs=1e-7)
    assert th[:-1].sum() == pytest.approx(1.3, rel=1e-10)      # P = sum K (Eq. 3)


def test_affine_invariances():
    """I -> aI + c gives K -> aK, B0 -> aB0 + c; R -> R + c gives B0 -> B0 - cP."""
    rng = np.random.default_rng(9)
    R = _star_ref((26, 26), 10, 1.3, rng)
    I = 0.8 * R + 12 + rng.normal(0, 1, R.shape)
    m = 5
    t = oracle.normal_solve(R, I, m)
    t2 = oracle.normal_solve(R, 2.5 * I + 7.0, m)
    np.testing.assert_allclose(t2[:-1], 2.5 * t[:-1], rtol=1e-9, atol=1e-10)
    assert t2[-1] == pytest.approx(2.5 * t[-1] + 7.0, rel=1e-9)
    t3 = oracle.normal_solve(R + 4.0, I, m)
    np.testing.assert_allclose(t3[:-1], t[:-1], rtol=1e-8, atol=1e-9)
    assert t3[-1] == pytest.approx(t[-1] - 4.0 * t[:-1].sum(), rel=1e-8)


def test_degenerate_constant_reference():
    R = np.full((12, 12), 3.0)
    I = np.random.default_rng(0).normal(size=(12, 12))
    with pytest.raises(oracle.Degenerate):
        oracle.normal_solve(R, I, 3)


# ---------------------------------------------------------------- Newton
def test_newton_from_far_lands_on_normal_solve():
    rng = np.random.default_rng(12)
    R = _star_ref((24, 24), 8, 1.4, rng)
    I = R * 1.2 + 3 + rng.normal(0, 1, R.shape)
    t_ne = oracle.normal_solve(R, I, 5)
    t_nw = oracle.newton(R, I, 5, np.zeros(26), LossSpec())
    # both are FP64 minima of the same quadratic: agree to the conditioning floor
    np.testing.assert_allclose(t_nw, t_ne, rtol=0, atol=1e-9 * np.max(np.abs(t_ne)))


@pytest.mark.parametrize("spec", [LossSpec("gauss", "ccd", sigma0=5, gain=1.5),
                                  LossSpec("huber", "ccd", sigma0=5, gain=1.5),
                                  LossSpec("gauss", "emccd", gain=0.5)],
                         ids=["ccd", "huber-ccd", "emccd"])
def test_newton_reaches_stationary_point(spec):
    rng = np.random.default_rng(13)
    R = _star_ref((30, 30), 10, 1.4, rng, flux=(500, 5000))
    I_nl = 1.05 * R + 150.0
    I = I_nl + rng.normal(0, 1, R.shape) * np.sqrt(25 + np.maximum(I_nl, 0) / 1.5)
    th = oracle.fit(R, I, 5, spec)
    _, g = oracle.loss_grad(R, I, 5, th, spec)
    _, g0 = oracle.loss_grad(R, I, 5, oracle.normal_solve(R, I, 5), spec)
    assert np.max(np.abs(g)) < 1e-8 * np.max(np.abs(g0))
    ev = np.linalg.eigvalsh(oracle.hessian(R, I, 5, th, spec))
    assert ev.min() > 0


# -------------------------------------------------------------- clipping
def test_sigma_clip_masks_planted_outlier_only():
    rng = np.random.default_rng(14)
    R = _star_ref((28, 28), 10, 1.4, rng)
    I = 1.1 * R + 4 + rng.normal(0, 1, R.shape)
    I[14, 15] += 500.0
    th = oracle.normal_solve(R, I, 5)
    mk = oracle.sigma_clip(R, I, 5, th, LossSpec(), kappa=5.0)
    bad = np.argwhere(mk == 0)
    assert [tuple(b) for b in bad] == [(14, 15)]
    th2, mk2 = oracle.fit_clipped(R, I, 5, LossSpec(), passes=2)
    assert mk2[14, 15] == 0
    I2 = I.copy()
    I2[14, 15] = 0.0
    np.testing.assert_allclose(th2, oracle.normal_solve(R, I2, 5, mask=mk2), rtol=1e-12)


# --------------------------------------------------- statistical (Sec. 3.3)
def test_mfv_of_weighted_fit_matches_paper_b08_value():
    """MFV of a correctly weighted 19x19 fit on a 142x142 S10-like pair falls
    in the band the paper prints for B08 (Sec. 3.3 table)."""
    from paper_2104_13715_gb300 import synth
    gold = GOLD["s10_mfv_b08_snr1_oversampled"]
    vals = []
    for seed in range(3):
        p = synth.PairSpec(size=(142, 142), n_stars=50, m=19, fwhm_ref=2.355 * 1.5,
                           kernel_sigma=1.5, sky=100.0, read=5.0, gain=1.0,
                           flux_law="paper")
        d = synth.make_pair(p, seed)
        I_nl = d["I_noiseless"].astype(np.float64)
        var = 25.0 + I_nl                      # Eq. 25, the true pixel variance
        th = oracle.normal_solve(d["R"], d["I"], 19, var=var)
        eps = oracle.diff_image(d["R"], d["I"], 19, th) / np.sqrt(_valid(var, 19))
        assert eps.size == GOLD["ndata_142_m19"]["value"]
        vals.append(np.var(eps, ddof=1))        # MFV (Eq. 30)
    med = float(np.median(vals))
    assert gold["median"] - 3 * (gold["median"] - gold["p16"]) < med < \
        gold["median"] + 3 * (gold["p84"] - gold["median"])


# --------------------------------------------------- regulariser (Sec. 2.7)
def _field(H, W, m, seed):
    """A star-field pair: I = R (*) K_true + B0 + noise, the valid region filled."""
    rng = np.random.default_rng(seed)
    R = _star_ref((H, W), 12, 1.5, rng) + 100.0
    yy, xx = np.mgrid[0:m, 0:m] - m // 2
    K = np.exp(-(xx ** 2 + yy ** 2) / (2 * 1.2 ** 2))
    K /= K.sum()
    th = np.append(K.ravel(), 30.0)
    I = np.full((H, W), 130.0)
    h = m // 2
    I[h:H - h, h:W - h] = _scipy_model(R, th, m) + rng.normal(0, 2.0, (H - 2 * h, W - 2 * h))
    return {"R": R, "I": I, "theta": th}


def test_laplacian_structure_and_quadratic_surface():
    """Eq. 21: symmetric, rows summing to zero (a constant kernel is not
    penalised), degree 2/3/4 at corners/edges/interior, B0 row and column zero;
    for the surface K[a, b] = a^2 + b^2 the discrete Laplacian is 4, so
    (L theta)_u = -4 at every interior pixel."""
    m = 5
    L = oracle.laplacian(m)
    n = m * m + 1
    assert L.shape == (n, n) and np.array_equal(L, L.T)
    assert np.allclose(L.sum(axis=1), 0.0)
    assert np.all(L[-1] == 0) and np.all(L[:, -1] == 0)
    deg = np.diag(L)[:-1].reshape(m, m)
    assert deg[0, 0] == 2 and deg[0, 2] == 3 and deg[2, 2] == 4
    a, b = np.mgrid[0:m, 0:m]
    th = np.append((a ** 2 + b ** 2).astype(float).ravel(), 7.0)
    Lth = (L @ th)[:-1].reshape(m, m)
    assert np.allclose(Lth[1:-1, 1:-1], -4.0)
    assert np.all(np.linalg.eigvalsh(L) > -1e-12)


def test_regularised_gradient_and_hessian_central_differences():
    m = 5
    d = _field(40, 36, m, seed=8)
    spec = oracle.LossSpec(rho="gauss", noise="ccd", sigma0=4.0, gain=1.3, var_floor=1e-6)
    rng = np.random.default_rng(8)
    th = np.full(m * m + 1, 1.0 / (m * m)) * (1 + 0.2 * rng.uniform(-1, 1, m * m + 1))
    th[-1] = float(np.median(d["I"]))
    lam = 3.0
    L0, g = oracle.loss_grad(d["R"], d["I"], m, th, spec, reg_lambda=lam)
    H = oracle.hessian(d["R"], d["I"], m, th, spec, reg_lambda=lam)
    for k in (0, 7, 12, m * m):
        e = np.zeros_like(th)
        e[k] = 1e-4 * max(1.0, abs(th[k]))
        Lp, gp = oracle.loss_grad(d["R"], d["I"], m, th + e, spec, reg_lambda=lam)
        Lm, gm = oracle.loss_grad(d["R"], d["I"], m, th - e, spec, reg_lambda=lam)
        assert (Lp - Lm) / (2 * e[k]) == pytest.approx(g[k], rel=1e-6, abs=1e-6 * np.max(np.abs(g)))
        np.testing.assert_allclose((gp - gm) / (2 * e[k]), H[:, k], rtol=1e-5,
                                   atol=1e-6 * np.max(np.abs(H)))


def test_regularised_normal_solve_is_stationary_and_smoother():
    """The regularised chi^2 minimum has zero regularised gradient, and a larger
    lam gives a kernel with a smaller Laplacian norm and a larger chi^2."""
    m = 7
    d = _field(60, 56, m, seed=9)
    spec = oracle.LossSpec()
    L = oracle.laplacian(m)
    prev = None
    for lam in (0.0, 1.0, 100.0):
        th = oracle.normal_solve(d["R"], d["I"], m, reg_lambda=lam)
        _, g = oracle.loss_grad(d["R"], d["I"], m, th, spec, reg_lambda=lam)
        scale = np.max(np.abs(oracle.loss_grad(d["R"], d["I"], m, np.zeros_like(th), spec)[1]))
        assert np.max(np.abs(g)) <= 1e-9 * scale
        rough = float(np.sum((L @ th) ** 2))
        chi2 = oracle.loss(d["R"], d["I"], m, th, spec)
        if prev is not None:
            assert rough < prev[0] and chi2 > prev[1]
        prev = (rough, chi2)


def test_penalty_is_the_squared_graph_laplacian_of_the_kernel_surface():
    """Eq. 20 written with array shifts instead of the matrix: (L theta)_u is
    the sum over the edge-neighbours v of u of (K_u - K_v); the penalty is
    lam * N_data * sum_u (L theta)_u^2 and B0 does not enter it."""
    m, lam, n_data = 6, 0.7, 1234
    rng = np.random.default_rng(5)
    K = rng.normal(size=(m, m))
    Lk = np.zeros((m, m))
    Lk[1:, :] += K[1:, :] - K[:-1, :]
    Lk[:-1, :] += K[:-1, :] - K[1:, :]
    Lk[:, 1:] += K[:, 1:] - K[:, :-1]
    Lk[:, :-1] += K[:, :-1] - K[:, 1:]
    th = np.append(K.ravel(), 99.0)
    v, g, Hp = oracle.penalty(th, m, lam, n_data)
    assert v == pytest.approx(lam * n_data * np.sum(Lk ** 2), rel=1e-12)
    assert g[-1] == 0 and np.all(Hp[-1] == 0)
    th2 = th.copy()
    th2[:-1] += 3.0              # a constant kernel offset is not penalised
    assert oracle.penalty(th2, m, lam, n_data)[0] == pytest.approx(v, rel=1e-12)
    d = _field(30, 28, 5, seed=2)
    t = d["theta"]
    L1, g1 = oracle.loss_grad(d["R"], d["I"], 5, t, reg_lambda=2.0)
    L0, g0 = oracle.loss_grad(d["R"], d["I"], 5, t)
    pv, pg, _ = oracle.penalty(t, 5, 2.0, oracle.ndata((30, 28), 5))
    assert L1 - L0 == pytest.approx(pv, rel=1e-9) and np.allclose(g1 - g0, pg, rtol=1e-9)


# ------------------------------------------- polynomial background (Sec. 2.6)
def test_background_basis_values_by_hand():
    """Eq. 18-19 at hand-worked pixels of a 9 x 13 image (m = 3, d = 2): the
    image centre (row 4, column 6) has eta = xi = 0; the first valid pixel
    (row 1, column 1) has eta = (1 - 6)/13, xi = (1 - 4)/9; the coefficient
    order is b_00, b_01, b_02, b_10, b_11, b_20 (power of xi fastest)."""
    Bs = oracle.background_basis((9, 13), 3, 2)
    assert Bs.shape == (7, 11, 6)
    np.testing.assert_allclose(Bs[3, 5], [1, 0, 0, 0, 0, 0], atol=0)
    eta, xi = -5.0 / 13.0, -1.0 / 3.0
    np.testing.assert_allclose(Bs[0, 0], [1, xi, xi * xi, eta, eta * xi, eta * eta],
                               rtol=1e-15)
    assert oracle.n_background(0) == 1 and oracle.n_background(3) == 10
    assert oracle.degree_of(np.zeros(9 + 6), 3) == 2
    with pytest.raises(ValueError):
        oracle.degree_of(np.zeros(9 + 5), 3)


def _poly_image(H, W, m, coef, deg):
    """Eq. 18 written directly over the valid region (row y, column x)."""
    h = m // 2
    y, x = np.mgrid[h:H - h, h:W - h].astype(float)
    eta, xi = (x - (W - 1) / 2) / W, (y - (H - 1) / 2) / H
    out = np.zeros_like(x)
    k = 0
    for p in range(deg + 1):
        for q in range(deg - p + 1):
            out += coef[k] * eta ** p * xi ** q
            k += 1
    return out


@pytest.mark.parametrize("deg", [0, 1, 3])
def test_model_is_correlation_plus_polynomial(deg):
    rng = np.random.default_rng(12 + deg)
    H, W, m = 17, 21, 5
    R = rng.normal(size=(H, W))
    nb = oracle.n_background(deg)
    th = rng.normal(size=m * m + nb)
    M = oracle.model(R, th, m)
    ref = _scipy_model(np.asarray(R), np.append(th[:m * m], 0.0), m) + \
        _poly_image(H, W, m, th[m * m:], deg)
    np.testing.assert_allclose(M, ref, rtol=0, atol=1e-12)


def test_polynomial_background_gradient_and_hessian_central_differences():
    m, deg = 5, 2
    d = _field(40, 44, m, seed=13)
    spec = oracle.LossSpec(rho="huber", noise="ccd", sigma0=4.0, gain=1.3, var_floor=1e-6)
    rng = np.random.default_rng(13)
    th = np.concatenate([np.full(m * m, 1.0 / (m * m)), [float(np.median(d["I"])), 3.0, -2.0,
                                                         5.0, 1.5, -4.0]])
    th[:m * m] *= 1 + 0.2 * rng.uniform(-1, 1, m * m)
    L0, g = oracle.loss_grad(d["R"], d["I"], m, th, spec)
    H = oracle.hessian(d["R"], d["I"], m, th, spec)
    assert g.shape == (m * m + 6,) and H.shape == (m * m + 6, m * m + 6)
    for k in (3, m * m, m * m + 1, m * m + 3, m * m + 5):
        e = np.zeros_like(th)
        e[k] = 1e-4 * max(1.0, abs(th[k]))
        Lp, gp = oracle.loss_grad(d["R"], d["I"], m, th + e, spec)
        Lm, gm = oracle.loss_grad(d["R"], d["I"], m, th - e, spec)
        assert (Lp - Lm) / (2 * e[k]) == pytest.approx(g[k], rel=1e-6, abs=1e-6 * np.max(np.abs(g)))
        np.testing.assert_allclose((gp - gm) / (2 * e[k]), H[:, k], rtol=1e-5,
                                   atol=1e-6 * np.max(np.abs(H)))


@pytest.mark.parametrize("deg", [1, 2, 3])
def test_normal_solve_recovers_an_injected_polynomial_background(deg):
    """Noiseless target I = R (x) K + B(x, y), B a degree-d polynomial written
    from Eq. 18 in the test: the normal solve of degree d returns K and every
    coefficient; a degree-0 fit of the same pair cannot."""
    rng = np.random.default_rng(20 + deg)
    H, W, m = 48, 52, 5
    R = _star_ref((H, W), 15, 1.4, rng) + 50.0
    yy, xx = np.mgrid[0:m, 0:m] - m // 2
    K = np.exp(-(xx ** 2 + yy ** 2) / 2.0)
    K *= 1.3 / K.sum()
    nb = oracle.n_background(deg)
    coef = rng.uniform(-40, 40, nb)
    coef[0] = 25.0
    I = np.zeros((H, W))
    h = m // 2
    I[h:H - h, h:W - h] = _scipy_model(R, np.append(K.ravel(), 0.0), m) + \
        _poly_image(H, W, m, coef, deg)
    th = oracle.normal_solve(R, I, m, deg=deg)
    np.testing.assert_allclose(th[:m * m], K.ravel(), rtol=0, atol=1e-9)
    np.testing.assert_allclose(th[m * m:], coef, rtol=0, atol=1e-7 * np.max(np.abs(coef)))
    th0 = oracle.normal_solve(R, I, m)
    assert np.max(np.abs(oracle.diff_image(R, I, m, th0))) > 1e-3
    assert np.max(np.abs(oracle.diff_image(R, I, m, th))) < 1e-8


# ------------------------------------------- spatially varying kernel (Sec. 1)
def _svk_direct(R, Ks, bg, m, dk, deg):
    """M by the definition, pixel by pixel: K_ab(x, y) = sum_c K_c[a][b] eta^p xi^q,
    then the correlation of that kernel with R, plus the background."""
    H, W = R.shape
    h = m // 2
    out = np.zeros((H - 2 * h, W - 2 * h))
    for y in range(H - 2 * h):
        for x in range(W - 2 * h):
            eta, xi = (x + h - (W - 1) / 2) / W, (y + h - (H - 1) / 2) / H
            Kxy = np.zeros((m, m))
            c = 0
            for p in range(dk + 1):
                for q in range(dk - p + 1):
                    Kxy += Ks[c] * eta ** p * xi ** q
                    c += 1
            B = 0.0
            c = 0
            for p in range(deg + 1):
                for q in range(deg - p + 1):
                    B += bg[c] * eta ** p * xi ** q
                    c += 1
            out[y, x] = np.sum(Kxy * R[y:y + m, x:x + m]) + B
    return out


@pytest.mark.parametrize("dk,deg", [(0, 0), (1, 0), (2, 1)])
def test_svk_model_is_the_pixel_by_pixel_definition(dk, deg):
    rng = np.random.default_rng(30 + dk)
    H, W, m = 17, 19, 5
    R = rng.normal(size=(H, W))
    nk, nb = oracle.n_background(dk), oracle.n_background(deg)
    th = rng.normal(size=nk * m * m + nb)
    Ks = [th[c * m * m:(c + 1) * m * m].reshape(m, m) for c in range(nk)]
    ref = _svk_direct(R, Ks, th[nk * m * m:], m, dk, deg)
    np.testing.assert_allclose(oracle.svk_model(R, th, m, dk), ref, rtol=0, atol=1e-12)


def test_svk_degree_zero_is_the_constant_kernel():
    m, deg = 5, 1
    d = _field(40, 44, m, seed=31)
    spec = oracle.LossSpec(rho="huber", noise="ccd", sigma0=4.0, gain=1.3, var_floor=1e-6)
    th = np.concatenate([d["theta"][:-1], [30.0, 2.0, -3.0]])
    np.testing.assert_allclose(oracle.svk_model(d["R"], th, m, 0), oracle.model(d["R"], th, m),
                               rtol=0, atol=1e-10)
    L1, g1 = oracle.svk_loss_grad(d["R"], d["I"], m, th, 0, spec)
    L0, g0 = oracle.loss_grad(d["R"], d["I"], m, th, spec)
    assert L1 == pytest.approx(L0, rel=1e-12)
    np.testing.assert_allclose(g1, g0, rtol=1e-9, atol=1e-9 * np.max(np.abs(g0)))
    np.testing.assert_allclose(oracle.svk_normal_solve(d["R"], d["I"], m, 0, deg=deg),
                               oracle.normal_solve(d["R"], d["I"], m, deg=deg), rtol=1e-8, atol=1e-10)


def test_svk_gradient_central_differences():
    m, dk = 5, 1
    d = _field(36, 40, m, seed=32)
    spec = oracle.LossSpec(rho="gauss", noise="ccd", sigma0=4.0, gain=1.3, var_floor=1e-6)
    rng = np.random.default_rng(32)
    K0 = d["theta"][:-1]
    th = np.concatenate([K0, 0.02 * rng.normal(size=m * m), 0.02 * rng.normal(size=m * m), [30.0]])
    L0, g = oracle.svk_loss_grad(d["R"], d["I"], m, th, dk, spec)
    for k in (3, m * m + 7, 2 * m * m + 12, 3 * m * m):
        e = np.zeros_like(th)
        e[k] = 1e-5 * max(1.0, abs(th[k]))   # the difference error falls as the step squared
        Lp, _ = oracle.svk_loss_grad(d["R"], d["I"], m, th + e, dk, spec)
        Lm, _ = oracle.svk_loss_grad(d["R"], d["I"], m, th - e, dk, spec)
        assert (Lp - Lm) / (2 * e[k]) == pytest.approx(g[k], rel=1e-6, abs=1e-6 * np.max(np.abs(g)))


def test_svk_normal_solve_recovers_an_injected_varying_kernel():
    """Noiseless target made pixel by pixel from a kernel whose width and centre
    drift linearly across the field (dk = 1) plus a tilted background: the dk = 1
    solve returns every coefficient; the constant-kernel solve cannot fit it."""
    rng = np.random.default_rng(33)
    H, W, m, dk, deg = 44, 48, 5, 1, 1
    R = _star_ref((H, W), 25, 1.3, rng) + 40.0
    yy, xx = np.mgrid[0:m, 0:m] - m // 2
    G = np.exp(-(xx ** 2 + yy ** 2) / 2.0)
    K00 = G / G.sum()
    K01 = 0.3 * (np.roll(K00, 1, axis=0) - K00)     # drift along y
    K10 = 0.2 * (K00 * (xx ** 2 - 1.0))             # width change along x
    bg = np.array([20.0, 3.0, -5.0])
    I = np.zeros((H, W))
    h = m // 2
    I[h:H - h, h:W - h] = _svk_direct(R, [K00, K01, K10], bg, m, dk, deg)
    th = oracle.svk_normal_solve(R, I, m, dk, deg=deg)
    truth = np.concatenate([K00.ravel(), K01.ravel(), K10.ravel(), bg])
    np.testing.assert_allclose(th, truth, rtol=0, atol=1e-8)
    th0 = oracle.svk_normal_solve(R, I, m, 0, deg=deg)
    assert np.max(np.abs(oracle.svk_model(R, th0, m, 0) - _valid(I, m))) > 1e-3


def test_svk_hessian_and_newton():
    """The spatially varying kernel's Hessian is the central difference of its
    gradient; Newton lands on the normal solve for chi^2 and on a stationary
    point of the CCD likelihood."""
    m, dk = 5, 1
    d = _field(36, 40, m, seed=34)
    spec = oracle.LossSpec(rho="gauss", noise="ccd", sigma0=4.0, gain=1.3, var_floor=1e-6)
    rng = np.random.default_rng(34)
    th = np.concatenate([d["theta"][:-1], 0.02 * rng.normal(size=2 * m * m), [30.0]])
    Hm = oracle.svk_hessian(d["R"], d["I"], m, th, dk, spec)
    for k in (2, m * m + 4, 2 * m * m + 9, 3 * m * m):
        e = np.zeros_like(th)
        e[k] = 1e-5 * max(1.0, abs(th[k]))
        _, gp = oracle.svk_loss_grad(d["R"], d["I"], m, th + e, dk, spec)
        _, gm = oracle.svk_loss_grad(d["R"], d["I"], m, th - e, dk, spec)
        np.testing.assert_allclose((gp - gm) / (2 * e[k]), Hm[:, k], rtol=1e-5,
                                   atol=1e-6 * np.max(np.abs(Hm)))
    chi2 = oracle.LossSpec()
    ref = oracle.svk_normal_solve(d["R"], d["I"], m, dk)
    got = oracle.svk_newton(d["R"], d["I"], m, th, dk, chi2)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-8 * np.max(np.abs(ref)))
    tn = oracle.svk_newton(d["R"], d["I"], m, ref, dk, spec)
    _, g = oracle.svk_loss_grad(d["R"], d["I"], m, tn, dk, spec)
    _, g0 = oracle.svk_loss_grad(d["R"], d["I"], m, th, dk, spec)
    assert np.max(np.abs(g)) <= 1e-9 * np.max(np.abs(g0))

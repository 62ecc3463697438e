"""Observed Fisher information and covariance (dia_fisher, Sec. 2.5) against the
FP64 oracle's exact Hessian sum_p l''(M_p) phi_p phi_p^T.

Tolerances: F element-wise within 1e-6 of max|F| for a fixed variance (the
per-pixel weight is 1/v) and 2e-5 for a model-dependent variance (l'' then
depends on z, computed from the float32 model image); the returned covariance
is the float64 inverse of the returned F (checked against numpy's inverse of
that F to 1e-7 relative) and its Cramer-Rao bounds (Eq. 17) agree with the
oracle's to 1e-3; the positive-definiteness flag agrees with the sign of the
smallest eigenvalue of the oracle's Hessian."""
import numpy as np
import pytest
import torch

import oracle
from tests._helpers import SPECS, field, ospec, theta_start

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nat():
    from paper_2104_13715_gb300 import native
    return native


def _dev(a, dt=torch.float32):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)


def _run(nat, d, m, spec, theta, mask=None, var=None):
    out = nat.fisher(_dev(d["R"]), _dev(d["I"]), m, _dev(theta, torch.float64),
                     nat.loss_spec(**spec), mask=_dev(mask, torch.uint8), var=_dev(var))
    H = oracle.hessian(d["R"], d["I"], m, theta, ospec(spec), mask=mask, var=var)
    return out["F"].cpu().numpy(), out["cov"].cpu().numpy(), out["info"], H


def _check_inverse_and_bounds(F, cov, info, H):
    n = F.shape[0]
    assert info["positive_definite"] == 1 and info["n"] == n
    ref_inv = np.linalg.inv(F)
    assert np.max(np.abs(cov - ref_inv)) <= 1e-7 * np.max(np.abs(ref_inv))
    sign, logdet = np.linalg.slogdet(F)
    assert sign > 0 and abs(info["log_det"] - logdet) <= 1e-8 * max(1.0, abs(logdet))
    # Cramer-Rao bounds and the photometric-scale variance 1' Sigma_KK 1 (Eq. 3)
    cov_o = np.linalg.inv(H)
    sig, sig_o = np.sqrt(np.diag(cov)), np.sqrt(np.diag(cov_o))
    assert np.max(np.abs(sig - sig_o) / sig_o) <= 1e-3
    one = np.ones(n - 1)
    vp, vp_o = one @ cov[:-1, :-1] @ one, one @ cov_o[:-1, :-1] @ one
    assert abs(vp - vp_o) <= 1e-3 * vp_o


def test_fixed_variance_chi2_at_normal_solution(nat):
    m = 7
    d = field(120, 110, m, seed=11)
    var = (25.0 + np.maximum(d["I"], 0)).astype(np.float32)
    rng = np.random.default_rng(11)
    mask = (rng.random(d["R"].shape) > 0.05).astype(np.uint8)
    theta = oracle.normal_solve(d["R"], d["I"], m, mask=mask, var=var)
    F, cov, info, H = _run(nat, d, m, SPECS["gauss-fixed"], theta, mask=mask, var=var)
    assert np.max(np.abs(F - H)) <= 1e-6 * np.max(np.abs(H))
    h = m // 2
    assert info["ndata"] == int(mask[h:-h, h:-h].sum())
    _check_inverse_and_bounds(F, cov, info, H)


@pytest.mark.parametrize("name", ["gauss-ccd", "gauss-emccd", "huber-ccd"])
def test_model_dependent_variance_at_the_optimum(nat, name):
    m = 9
    d = field(130, 124, m, seed=12)
    spec = SPECS[name]
    th0 = theta_start(m, d["I"])
    theta = oracle.newton(d["R"], d["I"], m, th0, ospec(spec))
    F, cov, info, H = _run(nat, d, m, spec, theta)
    assert np.max(np.abs(F - H)) <= 2e-5 * np.max(np.abs(H))
    if np.linalg.eigvalsh(H).min() > 0:
        _check_inverse_and_bounds(F, cov, info, H)


def test_indefinite_cauchy_hessian_raises_the_warning_flag(nat):
    """Far from the optimum many |z| > 1, where the Cauchy rho'' < 0: the
    Hessian is indefinite and the covariance is reported invalid (Sec. 2.5)."""
    m = 5
    d = field(90, 96, m, seed=13, scale=1.6, b0=300.0)
    spec = SPECS["cauchy-fixed"]
    theta = theta_start(m, d["I"])
    theta[-1] = 0.0
    F, cov, info, H = _run(nat, d, m, spec, theta)
    assert np.max(np.abs(F - H)) <= 2e-5 * np.max(np.abs(H))
    lam = np.linalg.eigvalsh(H)
    assert lam.min() < -1e-6 * lam.max()          # clearly indefinite
    assert info["positive_definite"] == 0
    assert np.all(np.isnan(cov))


def test_covariance_at_a_gpu_fit(nat):
    """The intended use: dia_fit, then dia_fisher at the fitted theta."""
    m = 11
    d = field(160, 150, m, seed=14)
    spec = SPECS["gauss-ccd"]
    R, I = _dev(d["R"]), _dev(d["I"])
    fit = nat.fit(R, I, m, nat.loss_spec(**spec), nat.default_opts())
    theta = fit["theta"].cpu().numpy()
    F, cov, info, H = _run(nat, d, m, spec, theta)
    assert np.max(np.abs(F - H)) <= 2e-5 * np.max(np.abs(H))
    _check_inverse_and_bounds(F, cov, info, H)

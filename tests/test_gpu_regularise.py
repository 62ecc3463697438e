"""Fits with the kernel regulariser of Sec. 2.7 (Eq. 20, Eq. 21) through the C
ABI against the FP64 oracle's regularised optimum.

Tolerances as for the unregularised fits: max |K - K*| <= 1e-4 |sum K*| and
|B0 - B0*| <= 1e-4 x sky."""
import numpy as np
import pytest
import torch

import oracle
from paper_2104_13715_gb300 import synth
from tests._helpers import SPECS, field, ospec

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nat():
    from paper_2104_13715_gb300 import native
    return native


def _t(a, dt=torch.float32):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)


def _check(theta, ref, sky, tol=1e-4):
    ek = np.max(np.abs(theta[:-1] - ref[:-1])) / abs(ref[:-1].sum())
    eb = abs(theta[-1] - ref[-1]) / sky
    assert ek <= tol and eb <= tol, (ek, eb)


@pytest.mark.parametrize("lam", [0.1, 10.0, 100.0])
@pytest.mark.parametrize("precond,adam", [(1, 5000), (1, 0), (0, 0)])
def test_regularised_chi2_matches_regularised_normal_equations(nat, lam, precond, adam):
    """(A + 2 lam N_data L^T L) theta = b, over the range of lambda of Sec. 2.7,
    with the Gauss-Newton and the diagonal preconditioner, with and without the
    Adam phase; the reported loss is the regularised objective."""
    d = synth.workload("stamp128_m11_chi2", seed=4)
    m, sky = d["m"], float(np.median(d["I"]))
    ref = oracle.normal_solve(d["R"], d["I"], m, reg_lambda=lam)
    opts = nat.default_opts(reg_lambda=lam, precond=precond, max_adam_iters=adam,
                            history=20 if precond else 100)
    out = nat.fit(_t(d["R"]), _t(d["I"]), m, nat.loss_spec(**d["loss"]), opts)
    th = out["theta"].cpu().numpy()
    assert out["info"]["status"] == 0
    _check(th, ref, sky)
    Lo, _ = oracle.loss_grad(d["R"], d["I"], m, th, ospec(d["loss"]), reg_lambda=lam)
    assert out["info"]["loss"] == pytest.approx(Lo, rel=1e-5)


def test_regularisation_smooths_the_kernel(nat):
    """Larger lambda: smaller |L theta|^2 of the fitted kernel and larger chi^2,
    the trade-off Eq. 20 sets; lambda = 0 is the unregularised fit."""
    d = synth.workload("stamp128_m11_chi2", seed=5)
    m = d["m"]
    Lm = oracle.laplacian(m)
    spec = nat.loss_spec(**d["loss"])
    prev = None
    for lam in (0.0, 1.0, 30.0):
        out = nat.fit(_t(d["R"]), _t(d["I"]), m, spec, nat.default_opts(reg_lambda=lam))
        th = out["theta"].cpu().numpy()
        rough = float(np.sum((Lm @ th) ** 2))
        chi2 = oracle.loss(d["R"], d["I"], m, th, ospec(d["loss"]))
        if prev is not None:
            assert rough < prev[0] and chi2 > prev[1]
        prev = (rough, chi2)


@pytest.mark.parametrize("name", ["gauss-ccd", "cauchy-emccd"])
def test_regularised_likelihood_fit_is_the_newton_optimum(nat, name):
    """Model-dependent variance and a robust loss with the regulariser: the
    fitted theta is a stationary point of the regularised FP64 objective."""
    m, lam = 9, 3.0
    d = field(150, 140, m, seed=33)
    spec = SPECS[name]
    out = nat.fit(_t(d["R"]), _t(d["I"]), m, nat.loss_spec(**spec),
                  nat.default_opts(reg_lambda=lam, max_adam_iters=0))
    th = out["theta"].cpu().numpy()
    assert out["info"]["status"] == 0
    ref = oracle.newton(d["R"], d["I"], m, th, ospec(spec), reg_lambda=lam)
    _check(th, ref, float(np.median(d["I"])))


@pytest.mark.parametrize("precond", [1, 0])
def test_regularised_batch_matches_per_pair_solutions(nat, precond):
    """dia_fit_batch with the regulariser: every pair (mixed kernel sides and
    sizes, so that N_data differs between pairs) at its own regularised
    normal-equation optimum."""
    lam = 5.0
    ds = [field(96 + 16 * i, 100 + 8 * i, m, seed=40 + i) for i, m in enumerate((5, 9, 13, 7))]
    ms = (5, 9, 13, 7)
    items = [dict(R=_t(d["R"]), I=_t(d["I"]), m=m) for d, m in zip(ds, ms)]
    opts = nat.default_opts(reg_lambda=lam, precond=precond, history=20 if precond else 100)
    out = nat.fit_batch(items, nat.loss_spec(**SPECS["gauss-fixed"]), opts)
    assert out["status"] == 0
    for d, m, th, info in zip(ds, ms, out["thetas"], out["infos"]):
        assert info["status"] == 0
        ref = oracle.normal_solve(d["R"], d["I"], m, reg_lambda=lam)
        _check(th.cpu().numpy(), ref, float(np.median(d["I"])))


def test_negative_or_nonfinite_lambda_is_rejected(nat):
    d = synth.workload("stamp128_m11_chi2", seed=0)
    spec = nat.loss_spec(**d["loss"])
    for bad in (-1.0, float("nan"), float("inf")):
        with pytest.raises(nat.DiaError):
            nat.fit(_t(d["R"]), _t(d["I"]), d["m"], spec, nat.default_opts(reg_lambda=bad))

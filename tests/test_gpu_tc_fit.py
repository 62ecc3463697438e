"""The tensor-core evaluation as the form of dia_loss_grad and dia_fit
(dia_set_eval_form(DIA_EVAL_TC)): the same kernels as dia_loss_grad_tc inside
the fit's captured optimiser iterations.  Checked against the FP64 oracle:
the evaluation within the split-precision bound of the tensor-core tests (here
its 1e-5 max-norm form at generic points), fitted kernels within 1e-4 of
sum K* and backgrounds within 1e-4 of the sky of the oracle's Newton optimum
(the tolerances of the float32 form)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2104_13715_gb300 import synth
from tests._helpers import SPECS, field, ospec, rel_inf, theta_start

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nat():
    from paper_2104_13715_gb300 import native
    yield native
    native.set_eval_form(native.EVAL_FP32)


def _t(a, dt=torch.float32):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)


def _lk(d):
    return {k: v for k, v in d["loss"].items()
            if k in ("rho", "noise", "sigma0", "gain", "excess", "huber_c", "var", "var_floor")}


def _ospec(d):
    lk = _lk(d)
    if lk.get("noise", "fixed") == "fixed":
        lk.pop("sigma0", None)
        lk.pop("gain", None)
    return ospec(lk)


def test_form_switch_and_workspace(nat):
    """The switch takes the two forms only; the workspace grows by the
    tensor-core regions for kernels it serves and not for m > 31."""
    assert nat.lib.dia_set_eval_form(3) == nat.DIA_ERR_ARG
    nat.set_eval_form(nat.EVAL_FP32)
    n32 = nat.lib.dia_workspace_size(1000, 1100, 1100, 25, 0, 0)
    n32_big = nat.lib.dia_workspace_size(1000, 1100, 1100, 33, 0, 0)
    nat.set_eval_form(nat.EVAL_TC)
    try:
        assert nat.get_eval_form() == nat.EVAL_TC
        ntc = nat.lib.dia_workspace_size(1000, 1100, 1100, 25, 0, 0)
        assert ntc >= n32 + 1024 * 1152 * 4     # the padded g map (976 -> 1024, 1076 -> 1152)
        assert nat.lib.dia_workspace_size(1000, 1100, 1100, 33, 0, 0) == n32_big
    finally:
        nat.set_eval_form(nat.EVAL_FP32)


@pytest.mark.parametrize("m,name", [(5, "gauss-ccd"), (17, "cauchy-fixed"), (29, "huber-fixed")])
def test_loss_grad_in_the_tc_form_equals_the_tc_entry(nat, m, name):
    """dia_loss_grad under DIA_EVAL_TC runs the kernels of dia_loss_grad_tc
    (same partial sums, same reduction order) and both meet the oracle."""
    spec = SPECS[name]
    d = field(300, 420, m, seed=90 + m)
    rng = np.random.default_rng(m)
    var = rng.uniform(50, 400, d["R"].shape).astype(np.float32) if spec["noise"] == "fixed" else None
    mask = (rng.random(d["R"].shape) > 0.05).astype(np.uint8)
    th = theta_start(m, d["I"], rng, jitter=0.3)
    args = (_t(d["R"]), _t(d["I"]), m, torch.from_numpy(th), nat.loss_spec(**spec))
    kw = dict(mask=_t(mask, torch.uint8), var=_t(var))
    L1, g1 = nat.loss_grad_tc(*args, **kw)
    nat.set_eval_form(nat.EVAL_TC)
    try:
        L2, g2 = nat.loss_grad(*args, **kw)
    finally:
        nat.set_eval_form(nat.EVAL_FP32)
    assert L2.item() == L1.item()
    np.testing.assert_array_equal(g2.cpu().numpy(), g1.cpu().numpy())
    Lo, go = oracle.loss_grad(d["R"], d["I"], m, th, ospec(spec), mask=mask, var=var)
    assert rel_inf(g2.cpu().numpy(), go) <= 1e-5
    assert L2.item() == pytest.approx(Lo, rel=1e-5)


def test_ccd_fit_in_the_tc_form_matches_oracle_newton(nat):
    """1024^2, m = 19, CCD NLL: the fit with every evaluation on the tensor
    cores (many tiles per CTA, the converged graph iterations skipped by the
    kernels' done flag) against the FP64 Newton optimum from its result."""
    d = synth.workload("ccd1024_m19_nll", seed=0)
    m = d["m"]
    nat.set_eval_form(nat.EVAL_TC)
    try:
        out = nat.fit(_t(d["R"]), _t(d["I"]), m, nat.loss_spec(**_lk(d)))
    finally:
        nat.set_eval_form(nat.EVAL_FP32)
    assert out["info"]["status"] == 0, out["info"]
    th = out["theta"].cpu().numpy()
    ref = oracle.newton(d["R"], d["I"], m, th, _ospec(d))
    sky = float(np.median(d["I"]))
    ek = np.max(np.abs(th[:-1] - ref[:-1])) / abs(ref[:-1].sum())
    eb = abs(th[-1] - ref[-1]) / sky
    assert ek <= 1e-4 and eb <= 1e-4, (ek, eb)


def test_cauchy_clipped_fit_in_the_tc_form_matches_oracle_newton(nat):
    """The headline recipe at 2048^2 (Cauchy loss, 2 % masked, variance map,
    three sigma-clipped refits, m = 25) with tensor-core evaluations: the
    refits read the working mask; K, B0 and the difference image against the
    oracle's optimum on the mask the fit returns."""
    d = synth.workload("ccd4096_m25_cauchy_clip3", seed=0, size=2048)
    m = d["m"]
    opts = nat.default_opts(clip_passes=3, clip_kappa=5.0)
    nat.set_eval_form(nat.EVAL_TC)
    try:
        out = nat.fit(_t(d["R"]), _t(d["I"]), m, nat.loss_spec(**_lk(d)), opts,
                      mask=_t(d["mask"], torch.uint8), var=_t(d["var"]), want_mask=True,
                      want_diff=True)
    finally:
        nat.set_eval_form(nat.EVAL_FP32)
    assert out["info"]["status"] == 0 and out["info"]["clip_passes_done"] == 3, out["info"]
    th = out["theta"].cpu().numpy()
    mk = out["mask"].cpu().numpy()
    assert np.all(mk <= d["mask"])
    ref = oracle.newton(d["R"], d["I"], m, th, _ospec(d), mask=mk, var=d["var"], max_iter=2)
    sky = float(np.median(d["I"]))
    ek = np.max(np.abs(th[:-1] - ref[:-1])) / abs(ref[:-1].sum())
    eb = abs(th[-1] - ref[-1]) / sky
    D_ref = oracle.diff_image(d["R"], d["I"], m, ref)
    eD = np.max(np.abs(out["diff"].cpu().numpy() - D_ref)) / np.max(np.abs(d["I"]))
    assert ek <= 1e-4 and eb <= 1e-4 and eD <= 1e-5, (ek, eb, eD)


def test_unsupported_pairs_keep_the_float32_form(nat):
    """A polynomial background is outside the tensor-core form: dia_loss_grad
    under DIA_EVAL_TC gives the float32 form's result."""
    m = 9
    d = field(200, 240, m, seed=4)
    th = np.append(theta_start(m, d["I"]), [0.5, -0.3])   # B0 + two linear terms
    spec = nat.loss_spec(**SPECS["gauss-ccd"])
    L0, g0 = nat.loss_grad(_t(d["R"]), _t(d["I"]), m, torch.from_numpy(th), spec, bg_degree=1)
    nat.set_eval_form(nat.EVAL_TC)
    try:
        L1, g1 = nat.loss_grad(_t(d["R"]), _t(d["I"]), m, torch.from_numpy(th), spec, bg_degree=1)
    finally:
        nat.set_eval_form(nat.EVAL_FP32)
    assert L1.item() == L0.item()
    np.testing.assert_array_equal(g1.cpu().numpy(), g0.cpu().numpy())


@pytest.mark.parametrize("m,expect_tc", [(15, False), (19, True)])
def test_auto_form_picks_the_tensor_cores_from_m_19(nat, m, expect_tc):
    """DIA_EVAL_AUTO: dia_loss_grad gives the tensor-core entry's result
    bit for bit at m = 19 and the float32 form's at m = 15."""
    spec = nat.loss_spec(**SPECS["gauss-ccd"])
    d = field(260, 300, m, seed=7 * m)
    th = theta_start(m, d["I"], np.random.default_rng(m), jitter=0.2)
    args = (_t(d["R"]), _t(d["I"]), m, torch.from_numpy(th), spec)
    L_tc, g_tc = nat.loss_grad_tc(*args)
    L_32, g_32 = nat.loss_grad(*args)
    nat.set_eval_form(nat.EVAL_AUTO)
    try:
        L, g = nat.loss_grad(*args)
    finally:
        nat.set_eval_form(nat.EVAL_FP32)
    Le, ge = (L_tc, g_tc) if expect_tc else (L_32, g_32)
    assert L.item() == Le.item()
    np.testing.assert_array_equal(g.cpu().numpy(), ge.cpu().numpy())

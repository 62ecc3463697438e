"""Failure paths of dia_fit, all raised on the host or by the optimiser's own
status (no GPU fault is involved): the wall-clock polling limit, the
evaluation cap, non-finite pixels, an all-masked image; after each, the same
workspace fits normally again."""
import numpy as np
import pytest
import torch

import oracle
from tests._helpers import SPECS, field

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nat():
    from paper_2104_13715_gb300 import native
    return native


def _dev(a, dt=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)


@pytest.fixture(scope="module")
def pair():
    m = 9
    d = field(120, 110, m, seed=21)
    return d, m


def _ok_fit(nat, d, m, ws):
    out = nat.fit(_dev(d["R"]), _dev(d["I"]), m, nat.loss_spec(**SPECS["gauss-fixed"]),
                  nat.default_opts(), ws=ws)
    ref = oracle.normal_solve(d["R"], d["I"], m)
    th = out["theta"].cpu().numpy()
    assert out["status"] == nat.DIA_OK
    assert np.max(np.abs(th[:-1] - ref[:-1])) <= 1e-4 * abs(ref[:-1].sum())


def test_timeout_then_recovery(nat, pair):
    d, m = pair
    ws = nat.workspace(*d["R"].shape, m)
    out = nat.fit(_dev(d["R"]), _dev(d["I"]), m, nat.loss_spec(**SPECS["gauss-fixed"]),
                  nat.default_opts(timeout_s=1e-9, graph_iters=1), ws=ws, check=False)
    assert out["status"] == nat.DIA_ERR_TIMEOUT
    _ok_fit(nat, d, m, ws)


def test_evaluation_cap_returns_the_last_theta(nat, pair):
    d, m = pair
    ws = nat.workspace(*d["R"].shape, m)
    out = nat.fit(_dev(d["R"]), _dev(d["I"]), m, nat.loss_spec(**SPECS["gauss-fixed"]),
                  nat.default_opts(max_evals=7), ws=ws, check=False)
    assert out["status"] == nat.DIA_ERR_MAXITER
    assert out["info"]["evals"] == 7
    assert np.all(np.isfinite(out["theta"].cpu().numpy()))
    _ok_fit(nat, d, m, ws)


def test_nonfinite_pixel_is_reported(nat, pair):
    d, m = pair
    I = d["I"].copy()
    I[50, 50] = np.nan
    ws = nat.workspace(*d["R"].shape, m)
    out = nat.fit(_dev(d["R"]), _dev(I), m, nat.loss_spec(**SPECS["gauss-fixed"]),
                  nat.default_opts(), ws=ws, check=False)
    assert out["status"] == nat.DIA_ERR_NONFINITE
    assert out["info"]["reason"] == 7
    # masking the bad pixel makes the same pair fit
    mask = np.ones_like(I, dtype=np.uint8)
    mask[50, 50] = 0
    I2 = I.copy()
    I2[50, 50] = 0.0
    out = nat.fit(_dev(d["R"]), _dev(I2), m, nat.loss_spec(**SPECS["gauss-fixed"]),
                  nat.default_opts(), mask=_dev(mask, torch.uint8), ws=ws)
    assert out["status"] == nat.DIA_OK


def test_all_masked_is_degenerate(nat, pair):
    d, m = pair
    ws = nat.workspace(*d["R"].shape, m)
    mask = np.zeros(d["R"].shape, dtype=np.uint8)
    out = nat.fit(_dev(d["R"]), _dev(d["I"]), m, nat.loss_spec(**SPECS["gauss-fixed"]),
                  nat.default_opts(), mask=_dev(mask, torch.uint8), ws=ws, check=False)
    assert out["status"] == nat.DIA_ERR_DEGENERATE
    _ok_fit(nat, d, m, ws)

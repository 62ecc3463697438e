"""The simulated-image accuracy study of Sec. 3.2-3.3 at a reduced number of
simulations: pairs drawn by the paper's recipe, fitted in one dia_fit_batch
call with the CCD negative log-likelihood (sigma0 = 5, G = 1) and a 19x19
kernel, binned by SNR and sampling regime; the medians of P and MFV (and, with
its wide spread, MSE) in each well-populated bin agree with the paper's
PyTorchDIA values within three standard errors of a median,
1.2533 x (half the 16-84 % width the paper prints) / sqrt(n)."""
import json
import os

import numpy as np
import pytest
import torch

from paper_2104_13715_gb300 import synth

pytestmark = pytest.mark.gpu

TABLE = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "s10_table.json")))
N_SIM = 400
MIN_BIN = 25


@pytest.fixture(scope="module")
def study():
    from paper_2104_13715_gb300 import native as nat
    ds = [d for d in (synth.s10_pair(s) for s in range(N_SIM)) if d["snr_regime"] > 0]
    items = [dict(R=torch.from_numpy(d["R"]).cuda(), I=torch.from_numpy(d["I"]).cuda(), m=d["m"])
             for d in ds]
    spec = nat.loss_spec(rho="gauss", noise="ccd", sigma0=synth.S10_SIGMA0, gain=1.0,
                         var_floor=1e-6)
    out = nat.fit_batch(items, spec, nat.default_opts(), want_diff=True)
    rows = []
    for d, th, D, info in zip(ds, out["thetas"], out["diffs"], out["infos"]):
        assert info["status"] == 0, info
        met = synth.s10_metrics(d, th.cpu().numpy(), D.cpu().numpy())
        rows.append((d["snr_regime"], d["sampling"], met))
    return rows


def _bins(rows):
    b = {}
    for snr, samp, met in rows:
        b.setdefault((snr, samp), []).append(met)
    return {k: v for k, v in b.items() if len(v) >= MIN_BIN}


@pytest.mark.parametrize("metric,ours_key", [("P", "P"), ("MFV", "MFV"), ("MSE", "MSE_noisy")])
def test_medians_match_the_paper(study, metric, ours_key):
    """The paper's tabulated MSE (about 530-630, the mean pixel variance of the
    target) follows the mean squared residual against the noisy target, not
    the noiseless-target definition printed beside it (which gives ~15-30 for
    these fits): the table is compared with that quantity."""
    bins = _bins(study)
    assert len(bins) >= 3, {k: len(v) for k, v in bins.items()}
    for (snr, samp), mets in bins.items():
        med, lo, hi = TABLE[metric][str(snr)][samp]
        se = 1.2533 * 0.5 * (lo + hi) / np.sqrt(len(mets))
        ours = float(np.median([x[ours_key] for x in mets]))
        assert abs(ours - med) <= 3.0 * se, (metric, snr, samp, len(mets), ours, med, se)


def test_mse_against_the_noiseless_target_is_far_below_the_noise(study):
    """The printed definition of MSE (model against the noiseless target) is a
    small fraction of the pixel variance: its median is a few per cent of the
    median noisy-target residual (the model error of a 19x19 fit to ~15,000
    noisy pixels)."""
    ratio = np.array([met["MSE"] / met["MSE_noisy"] for _, _, met in study])
    assert np.median(ratio) < 0.1


def test_mfv_below_one_by_the_fitted_parameters(study):
    """Every fit removes about (m^2 + 1) degrees of freedom from N_data = 15376
    residuals: MFV clusters just under one (Sec. 3.3)."""
    mfv = np.array([met["MFV"] for _, _, met in study])
    assert 0.95 < np.median(mfv) < 1.0

"""The simulated-pair recipe of the accuracy study (Sec. 3.2) and its fit-quality
metrics (Sec. 3.3, Eq. 26-30), on the CPU: properties the paper's steps fix."""
import math

import numpy as np
import pytest

from paper_2104_13715_gb300 import synth


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_pair_follows_the_recipe(seed):
    d = synth.s10_pair(seed)
    assert d["R"].shape == d["I"].shape == (142, 142) and d["m"] == 19
    assert 0.5 <= d["phi_r"] <= 2.5 and 0.5 <= d["phi_k"] <= 2.5           # steps i, viii
    Inl = d["I_noiseless"]
    # step ix: sigma_I^2 = sigma0^2 + I_noiseless (sigma0 = 5, G = 1, F = 1)
    np.testing.assert_allclose(d["sigma_I"] ** 2, 25.0 + Inl, rtol=1e-12)
    # step v: skies ~ U(10, 1000); the noiseless images never fall below them
    assert 10.0 <= d["sky_i"] <= 1000.0 and 10.0 <= d["sky_r"] <= 1000.0
    assert Inl.min() >= d["sky_i"] and d["R_noiseless"].min() >= d["sky_r"]
    # step viii: the same stars, flux unchanged (P = 1): equal total star light up to
    # the flux the PSF wings carry past the edges
    fr = np.sum(d["R_noiseless"] - d["sky_r"])
    fi = np.sum(Inl - d["sky_i"])
    assert fi == pytest.approx(fr, rel=0.05)
    # brightest star at the centre (step iii): the noiseless target peaks there
    c = np.unravel_index(np.argmax(Inl), Inl.shape)
    assert abs(c[0] - 70.5) <= 1.5 and abs(c[1] - 70.5) <= 1.5
    # SNR_I of Eq. 25 and its regime
    snr = np.sum(Inl - d["sky_i"]) / math.sqrt(np.sum(d["sigma_I"] ** 2))
    assert d["snr"] == pytest.approx(snr, rel=1e-12)
    e = synth.S10_SNR_EDGES
    want = 1 if e[0] < d["snr"] < e[1] else 2 if e[1] < d["snr"] < e[2] else 3 if e[2] < d["snr"] < e[3] else 0
    assert d["snr_regime"] == want
    samp = (0 if d["phi_k"] > 1 else 1) if d["phi_r"] > 1 else (2 if d["phi_k"] > 1 else 3)
    assert d["sampling"] == samp
    # the reference is background subtracted (median 0)
    assert abs(float(np.median(d["R"]))) < 1e-3


def test_noise_levels_of_reference_and_target():
    """Steps vi-x: the target's normalised noise (I - I_noiseless)/sigma_I and the
    reference's (R - R_noiseless)/sigma_R, sigma_R^2 = 0.1 (25 + R_noiseless), are
    unit normal (the reference has ten times less variance)."""
    z = []
    for seed in range(6):
        d = synth.s10_pair(seed)
        z.append(((d["I"].astype(np.float64) - d["I_noiseless"]) / d["sigma_I"]).ravel())
    z = np.concatenate(z)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01
    zr = []
    for seed in range(6):
        d = synth.s10_pair(seed)
        sig_r = math.sqrt(0.1) * np.sqrt(25.0 + d["R_noiseless"])
        # R is returned median-subtracted: put the offset back before comparing
        r = d["R"].astype(np.float64)
        off = np.median(r - d["R_noiseless"])
        zr.append(((r - off - d["R_noiseless"]) / sig_r).ravel())
    zr = np.concatenate(zr)
    assert abs(zr.std() - 1.0) < 0.02


def test_metrics_definitions():
    """Eq. 26-30 on a hand-made case: a model off by a constant c gives
    MSE = c^2 against the noiseless target, MFB = -c/sigma and MFV = the
    variance of the noise in sigma units; P = sum K."""
    rng = np.random.default_rng(0)
    H = W = 40
    m = 3
    Inl = np.full((H, W), 100.0)
    sig = np.full((H, W), 2.0)
    noise = rng.normal(0, 1, (H, W)) * sig
    I = (Inl + noise).astype(np.float32)
    d = {"m": m, "I": I, "I_noiseless": Inl, "sigma_I": sig}
    c = 0.5
    h = m // 2
    M = Inl[h:-h, h:-h] + c
    D = I[h:-h, h:-h].astype(np.float64) - M
    th = np.append(np.full(m * m, 0.1), 0.0)
    met = synth.s10_metrics(d, th, D)
    assert met["P"] == pytest.approx(0.9)
    assert met["MSE"] == pytest.approx(c * c, rel=1e-9)
    eps = (noise[h:-h, h:-h] - c) / 2.0
    assert met["MFB"] == pytest.approx(eps.mean(), abs=1e-6)
    assert met["MFV"] == pytest.approx(eps.var(ddof=1), rel=1e-6)
    assert met["MSE_noisy"] == pytest.approx(np.mean(D * D), rel=1e-9)


def test_regime_populations_follow_the_paper_counts():
    """The paper prints how its 71,569 simulations fall into the 3 SNR x 4
    sampling bins (Sec. 3.3 table).  The recipe's draws fall into the bins in
    the same proportions: each bin's share within 4 binomial standard errors
    (1,500 draws)."""
    import json
    import os
    table = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "s10_table.json")))
    counts = {(int(r), s): n for r, row in table["N_sim"].items() for s, n in enumerate(row)}
    total = sum(counts.values())
    draws = [synth.s10_pair(seed) for seed in range(1500)]
    inside = [(d["snr_regime"], d["sampling"]) for d in draws if d["snr_regime"] > 0]
    n = len(inside)
    assert n > 900
    for key, c in counts.items():
        p = c / total
        got = sum(1 for k in inside if k == key) / n
        se = math.sqrt(p * (1 - p) / n)
        assert abs(got - p) <= 4 * se + 1e-3, (key, got, p)


def test_per_star_psf_widths_and_a_varying_target():
    """render_stars with one width per star equals the sum of single renders;
    a target PSF that widens with eta (the input of the spatially varying
    kernel tests) keeps each star's flux and widens the stars on the right."""
    rng = np.random.default_rng(0)
    xs, ys = rng.uniform(10, 50, 5), rng.uniform(10, 50, 5)
    fl, sg = rng.uniform(100, 1000, 5), rng.uniform(0.8, 2.0, 5)
    one = synth.render_stars((64, 64), xs, ys, fl, sg)
    parts = sum(synth.render_stars((64, 64), xs[i:i + 1], ys[i:i + 1], fl[i:i + 1], sg[i])
                for i in range(5))
    np.testing.assert_allclose(one, parts, rtol=1e-9, atol=1e-4)   # window truncation at 6 sigma
    np.testing.assert_allclose(one.sum(), fl.sum(), rtol=1e-6)
    base = dict(size=(64, 200), n_stars=2, m=5, fwhm_ref=2.0, kernel_sigma=1.0, ref_noise=False,
                read=0.0, sky=0.0)
    flat = synth.make_pair(synth.PairSpec(**base), 3)["I_noiseless"]
    var = synth.make_pair(synth.PairSpec(**base, kernel_sigma_slope=(1.5, 0.0)), 3)["I_noiseless"]
    np.testing.assert_allclose(var.sum(), flat.sum(), rtol=1e-6)
    # the widths differ from the constant-PSF render only through eta: a star
    # rendered alone at the right edge is wider (lower peak) than at the left
    W = 200
    left = synth.render_stars((64, W), [20.0], [32.0], [1000.0], 1.0)
    sl = np.sqrt(synth.fwhm_to_sigma(2.0) ** 2 + (1.0 + 1.5 * (20.0 - 0.5 * (W - 1)) / W) ** 2)
    sr = np.sqrt(synth.fwhm_to_sigma(2.0) ** 2 + (1.0 + 1.5 * (180.0 - 0.5 * (W - 1)) / W) ** 2)
    assert sl < sr
    assert synth.render_stars((64, W), [180.0], [32.0], [1000.0], sr).max() < \
        synth.render_stars((64, W), [20.0], [32.0], [1000.0], sl).max()
    assert not np.allclose(var, flat)

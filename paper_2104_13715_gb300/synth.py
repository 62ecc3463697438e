"""Seeded synthetic star-field pairs (reference R, target I) for tests and benchmarks.

This module renders inputs only: star fields with pixel-integrated Gaussian
PSFs, sky, Poisson and read noise, masks and outliers.  It contains none of the
fit's arithmetic (no convolution with a kernel, no loss): the target is rendered
directly with the PSF width phi_I^2 = phi_R^2 + phi_K^2 that a Gaussian kernel of
width phi_K produces (Sec. 3.1 step viii, Eq. 24), its stars scaled by the
photometric factor P and its sky set to P*S_R + B0.

The recipe follows the paper's simulated-image procedure (Sec. 3.1): uniform
sub-pixel star positions, a symmetric Gaussian PSF, a constant sky, a reference
with 10x less pixel variance than the target (Eq. 22-23), and a target with
variance sigma0^2 + I/G (Eq. 25-26).  The named workloads below set the
parameters (image side, star count, flux law, PSF widths, kernel side, loss).
The reference handed to the fit is background-subtracted by its median, as the
paper always does (Sec. 2.9).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy.special import erf


def fwhm_to_sigma(fwhm: float) -> float:
    return fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0)))


def render_stars(shape, xs, ys, fluxes, sigma, chunk: int = 20000) -> np.ndarray:
    """Sum of pixel-integrated, unit-normalised Gaussian profiles.

    Pixel (i, j) covers [j-0.5, j+0.5) x [i-0.5, i+0.5); star coordinates are
    continuous (x = column, y = row).  ``sigma``: one PSF width, or one per star."""
    H, W = shape
    img = np.zeros(H * W, dtype=np.float64)
    sig_all = np.broadcast_to(np.asarray(sigma, np.float64), (len(xs),))
    r = max(2, int(math.ceil(6.0 * float(np.max(sig_all)))) if len(xs) else 2)
    off = np.arange(-r, r + 1)
    for c0 in range(0, len(xs), chunk):
        x = np.asarray(xs[c0:c0 + chunk], np.float64)
        y = np.asarray(ys[c0:c0 + chunk], np.float64)
        f = np.asarray(fluxes[c0:c0 + chunk], np.float64)
        s2 = (sig_all[c0:c0 + chunk] * math.sqrt(2.0))[:, None]
        cx = np.floor(x + 0.5).astype(np.int64)[:, None] + off[None, :]
        cy = np.floor(y + 0.5).astype(np.int64)[:, None] + off[None, :]
        px = 0.5 * (erf((cx + 0.5 - x[:, None]) / s2) - erf((cx - 0.5 - x[:, None]) / s2))
        py = 0.5 * (erf((cy + 0.5 - y[:, None]) / s2) - erf((cy - 0.5 - y[:, None]) / s2))
        px = np.where((cx >= 0) & (cx < W), px, 0.0)
        py = np.where((cy >= 0) & (cy < H), py, 0.0)
        cxc = np.clip(cx, 0, W - 1)
        cyc = np.clip(cy, 0, H - 1)
        vals = f[:, None, None] * py[:, :, None] * px[:, None, :]
        idx = cyc[:, :, None] * W + cxc[:, None, :]
        img += np.bincount(idx.reshape(-1), weights=vals.reshape(-1), minlength=H * W)
    return img.reshape(H, W)


def add_noise(img, rng, gain: float, read: float, var_scale: float = 1.0) -> np.ndarray:
    """Poisson photon noise at gain G (e-/ADU) plus Gaussian read noise, with the
    total variance scaled by `var_scale` (0.1 for the stacked reference, Eq. 22)."""
    if var_scale == 1.0:
        e = rng.poisson(np.maximum(img, 0.0) * gain).astype(np.float64) / gain
        return e + rng.normal(0.0, read, img.shape)
    sd = math.sqrt(var_scale) * np.sqrt(read * read + np.maximum(img, 0.0) / gain)
    return img + rng.normal(0.0, 1.0, img.shape) * sd


@dataclass
class PairSpec:
    """Parameters of one synthetic reference/target pair."""
    size: tuple                      # (H, W)
    n_stars: int
    m: int                           # kernel side (odd)
    fwhm_ref: float                  # reference PSF FWHM (px)
    kernel_sigma: float              # phi_K of the injected Gaussian kernel (px)
    scale: float = 1.0               # photometric scale factor P (Eq. 3)
    b0: float = 0.0                  # differential background B0
    sky: float = 100.0               # reference sky S_R
    flux: tuple = (1e2, 1e5)         # flux range
    flux_law: str = "loguniform"     # or "paper": F^{-3/2} ~ U(1e-9, 10^-4.5)
    shift: tuple = (0.0, 0.0)        # sub-pixel shift of the target (dx, dy)
    gain: float = 1.0
    read: float = 5.0
    ref_noise: bool = True           # reference with 10x less variance (Eq. 22-23)
    mask_frac: float = 0.0           # Bernoulli fraction of bad (masked) pixels
    cosmic_frac: float = 0.0         # unmasked outliers, +U(1e3, 1e4)
    # a target PSF that changes over the image (what a spatially varying kernel
    # fits): phi_K + a_x eta + a_y xi and a shift (dx, dy) + (b_x eta, b_y xi),
    # eta, xi the star's normalised coordinates (x - (W-1)/2)/W, (y - (H-1)/2)/H
    kernel_sigma_slope: tuple = (0.0, 0.0)
    shift_slope: tuple = (0.0, 0.0)
    loss: dict = field(default_factory=dict)


def make_pair(spec: PairSpec, seed: int) -> dict:
    """Render one pair.  Returns float32 images (R background-subtracted), an
    optional uint8 mask (1 = use) and fixed-variance map, and the truth."""
    rng = np.random.default_rng(seed)
    H, W = spec.size
    n = spec.n_stars
    xs = rng.uniform(-0.5, W - 0.5, n)
    ys = rng.uniform(-0.5, H - 0.5, n)
    if spec.flux_law == "paper":
        u = rng.uniform(1e-9, 10 ** -4.5, n)
        fl = u ** (-2.0 / 3.0)
    else:
        lo, hi = spec.flux
        fl = np.exp(rng.uniform(math.log(lo), math.log(hi), n))
    sr = fwhm_to_sigma(spec.fwhm_ref)
    eta = (xs - 0.5 * (W - 1)) / W
    xi = (ys - 0.5 * (H - 1)) / H
    sk = spec.kernel_sigma + spec.kernel_sigma_slope[0] * eta + spec.kernel_sigma_slope[1] * xi
    si = np.sqrt(sr * sr + sk ** 2)
    R_nl = spec.sky + render_stars((H, W), xs, ys, fl, sr)
    I_nl = (spec.scale * spec.sky + spec.b0) + render_stars(
        (H, W), xs + spec.shift[0] + spec.shift_slope[0] * eta,
        ys + spec.shift[1] + spec.shift_slope[1] * xi, fl * spec.scale, si)
    R = add_noise(R_nl, rng, spec.gain, spec.read, 0.1) if spec.ref_noise else R_nl.copy()
    I = add_noise(I_nl, rng, spec.gain, spec.read)
    mask = None
    if spec.mask_frac > 0:
        mask = (rng.random((H, W)) >= spec.mask_frac).astype(np.uint8)
    if spec.cosmic_frac > 0:
        hit = rng.random((H, W)) < spec.cosmic_frac
        I = I + hit * rng.uniform(1e3, 1e4, (H, W))
    sky_ref = float(np.median(R))
    out = dict(
        R=(R - sky_ref).astype(np.float32),
        I=I.astype(np.float32),
        mask=mask,
        m=spec.m,
        loss=dict(spec.loss),
        truth=dict(scale=spec.scale, b0=spec.b0, kernel_sigma=spec.kernel_sigma,
                   sky_ref=sky_ref, b0_subtracted=spec.b0 + spec.scale * sky_ref),
        I_noiseless=I_nl.astype(np.float32),
        seed=seed,
    )
    if spec.loss.get("var_map") == "target":
        # fixed per-pixel variance estimated from the target itself
        g = spec.loss.get("gain", 1.0)
        s0 = spec.loss.get("sigma0", 0.0)
        out["var"] = (s0 * s0 + np.maximum(I, 0.0) / g).astype(np.float32)
    return out


# ---------------------------------------------------------------------------
# Named workloads.  Loss dicts use plain keys shared by the oracle and the
# binding: rho (gauss|huber|cauchy), noise (fixed|ccd|emccd), sigma0, gain,
# excess, huber_c, var (scalar fixed variance), var_floor; clip passes and
# kappa for the sigma-clipped refits.
# ---------------------------------------------------------------------------

WORKLOADS = {
    # 128^2 stamp, 200 stars, 11x11 kernel, fixed-variance chi^2
    "stamp128_m11_chi2": PairSpec(
        size=(128, 128), n_stars=200, m=11, fwhm_ref=2.0, kernel_sigma=1.2,
        scale=1.15, b0=40.0, sky=100.0, flux=(1e2, 1e5), read=5.0, gain=1.0,
        loss=dict(rho="gauss", noise="fixed", var=1.0)),
    # 1024^2, 5,000 stars, 19x19 kernel, CCD negative log-likelihood
    "ccd1024_m19_nll": PairSpec(
        size=(1024, 1024), n_stars=5000, m=19, fwhm_ref=2.5,
        kernel_sigma=math.sqrt(fwhm_to_sigma(4.0) ** 2 - fwhm_to_sigma(2.5) ** 2),
        shift=(0.3, 0.3), scale=1.0, b0=0.0, sky=100.0, read=6.0, gain=1.5,
        loss=dict(rho="gauss", noise="ccd", sigma0=6.0, gain=1.5, var_floor=1e-6)),
    # 4096^2 crowded field, 60,000 stars, 25x25 kernel, Cauchy loss with
    # 2% masked pixels, 0.1% cosmic rays and 3 sigma-clipped refits
    "ccd4096_m25_cauchy_clip3": PairSpec(
        size=(4096, 4096), n_stars=60000, m=25, fwhm_ref=2.0,
        kernel_sigma=math.sqrt(fwhm_to_sigma(3.6) ** 2 - fwhm_to_sigma(2.0) ** 2),
        scale=1.0, b0=20.0, sky=100.0, read=5.0, gain=1.0,
        mask_frac=0.02, cosmic_frac=0.001,
        loss=dict(rho="cauchy", noise="fixed", var_map="target", sigma0=5.0, gain=1.0,
                  clip_passes=3, kappa=5.0)),
    # 4096^2 field with small kernels (3x3, 5x5), fixed-variance chi^2: the
    # memory-bound end of the fused kernel (a few flop per byte)
    "ccd4096_m3_chi2": PairSpec(
        size=(4096, 4096), n_stars=60000, m=3, fwhm_ref=2.0, kernel_sigma=0.5,
        scale=1.0, b0=20.0, sky=100.0, read=5.0, gain=1.0,
        loss=dict(rho="gauss", noise="fixed", var=1.0)),
    "ccd4096_m5_chi2": PairSpec(
        size=(4096, 4096), n_stars=60000, m=5, fwhm_ref=2.0, kernel_sigma=0.8,
        scale=1.0, b0=20.0, sky=100.0, read=5.0, gain=1.0,
        loss=dict(rho="gauss", noise="fixed", var=1.0)),
    # mid-size kernels on the same 4096^2 chi^2 field (kernel-side studies)
    "ccd4096_m9_chi2": PairSpec(
        size=(4096, 4096), n_stars=60000, m=9, fwhm_ref=2.0, kernel_sigma=1.2,
        scale=1.0, b0=20.0, sky=100.0, read=5.0, gain=1.0,
        loss=dict(rho="gauss", noise="fixed", var=1.0)),
    "ccd4096_m13_chi2": PairSpec(
        size=(4096, 4096), n_stars=60000, m=13, fwhm_ref=2.0, kernel_sigma=1.5,
        scale=1.0, b0=20.0, sky=100.0, read=5.0, gain=1.0,
        loss=dict(rho="gauss", noise="fixed", var=1.0)),
    # 2048^2 high-dynamic-range field, 21x21 kernel, CCD NLL
    "hdr2048_m21_nll": PairSpec(
        size=(2048, 2048), n_stars=15000, m=21, fwhm_ref=2.0,
        kernel_sigma=math.sqrt(fwhm_to_sigma(3.6) ** 2 - fwhm_to_sigma(2.0) ** 2),
        scale=1.0, b0=0.0, sky=2000.0, flux=(1e1, 1e6), read=5.0, gain=1.0,
        loss=dict(rho="gauss", noise="ccd", sigma0=5.0, gain=1.0, var_floor=1e-6)),
}


def workload(name: str, seed: int = 0, size=None) -> dict:
    """Render a named workload; `size` overrides the image side (star count
    scales with area) for reduced-size test cases of the same recipe."""
    spec = WORKLOADS[name]
    if size is not None:
        H, W = (size, size) if np.isscalar(size) else size
        area = (H * W) / (spec.size[0] * spec.size[1])
        spec = PairSpec(**{**spec.__dict__, "size": (H, W),
                           "n_stars": max(1, int(round(spec.n_stars * area)))})
    out = make_pair(spec, seed)
    out["name"] = name
    return out


def batch_specs(n_pairs: int = 512, seed: int = 0, side=(64, 512), m_range=(7, 21)):
    """Specs of the batched workload: uneven stamps (side ~ U{64..512}), odd
    kernel sides ~ U{7..21}, per-pair phi_K ~ U(0.5, 2.5) (Sec. 3.1 viii),
    P ~ U(0.8, 1.3), B0 ~ U(-50, 50), lg star density 1.5 per 100^2 px and
    phi_R = 1 (Sec. 5.2), the paper's F^{-3/2} flux law (Sec. 3.1 iii)."""
    rng = np.random.default_rng(10_000 + seed)
    odd = np.arange(m_range[0], m_range[1] + 1, 2)
    specs = []
    for _ in range(n_pairs):
        s = int(rng.integers(side[0], side[1] + 1))
        m = int(rng.choice(odd))
        specs.append(PairSpec(
            size=(s, s), n_stars=max(1, int(round(10 ** 1.5 * s * s / 1e4))), m=m,
            fwhm_ref=2.0 * math.sqrt(2 * math.log(2.0)) * 1.0,
            kernel_sigma=float(rng.uniform(0.5, 2.5)), scale=float(rng.uniform(0.8, 1.3)),
            b0=float(rng.uniform(-50, 50)), sky=100.0, flux_law="paper", read=5.0,
            gain=1.0, loss=dict(rho="gauss", noise="fixed", var=1.0)))
    return specs


def batch(n_pairs: int = 512, seed: int = 0, **kw) -> list:
    return [make_pair(s, 100_000 * (seed + 1) + k)
            for k, s in enumerate(batch_specs(n_pairs, seed, **kw))]


# ---------------------------------------------------------------------------
# The simulated pairs of the paper's accuracy study (Sec. 3.2, after the S10
# set of Bramich et al. 2016): 142 x 142 pixels, Gaussian PSFs and kernel,
# CCD noise with sigma0 = 5 ADU, G = 1, a reference with ten times less
# variance.  Star profiles are pixel-integrated unit Gaussians (the paper says
# only "normalised"); the target noise is Gaussian with the noise map of the
# noiseless target (the paper's step x).
# ---------------------------------------------------------------------------
S10_SIZE = 142
S10_M = 19
S10_SIGMA0 = 5.0
S10_SNR_EDGES = (8.0, 40.0, 200.0, 1000.0)   # SNR regimes 1, 2, 3 of the accuracy study


def s10_pair(seed: int, size: int = S10_SIZE) -> dict:
    """One simulated reference/target pair (Sec. 3.2 steps i-x).  Returns the
    background-subtracted float32 reference, the float32 target, the noiseless
    target, its noise map sigma_I, phi_R, phi_K, SNR_I and the regime labels
    (SNR regime 1-3 or 0 outside, sampling regime 0-3 = i-iv)."""
    rng = np.random.default_rng(seed)
    H = W = size
    phi_r = rng.uniform(0.5, 2.5)                         # (i)
    lg_rho = rng.uniform(0.0, 3.0)                         # (ii) per 100 x 100 px
    n = max(1, int(round(10 ** lg_rho * H * W / 1e4)))
    xs = rng.uniform(-0.5, W - 0.5, n)
    ys = rng.uniform(-0.5, H - 0.5, n)
    u = rng.uniform(1e-9, 10 ** -4.5, n)                   # (iii) F^-3/2 uniform
    fl = u ** (-2.0 / 3.0)
    b = int(np.argmax(fl))                                 # brightest star to the centre
    xs[b], ys[b] = 0.5 * (W - 1), 0.5 * (H - 1)
    s_r = rng.uniform(10.0, 1000.0)                        # (v)
    R_nl = s_r + render_stars((H, W), xs, ys, fl, phi_r)   # (iv)
    sig_r = math.sqrt(0.1) * np.sqrt(S10_SIGMA0 ** 2 + R_nl)          # (vi)
    R = R_nl + rng.normal(0.0, 1.0, (H, W)) * sig_r       # (vii)
    phi_k = rng.uniform(0.5, 2.5)                          # (viii)
    phi_i = math.sqrt(phi_r * phi_r + phi_k * phi_k)
    s_i = rng.uniform(10.0, 1000.0)
    dx, dy = rng.uniform(-0.5, 0.5, 2)
    I_nl = s_i + render_stars((H, W), xs + dx, ys + dy, fl, phi_i)
    sig_i = np.sqrt(S10_SIGMA0 ** 2 + I_nl)               # (ix)
    I = I_nl + rng.normal(0.0, 1.0, (H, W)) * sig_i       # (x)
    snr = float(np.sum(I_nl - s_i) / math.sqrt(float(np.sum(sig_i ** 2))))
    e = S10_SNR_EDGES
    snr_regime = 1 if e[0] < snr < e[1] else 2 if e[1] < snr < e[2] else 3 if e[2] < snr < e[3] else 0
    samp = (0 if phi_k > 1 else 1) if phi_r > 1 else (2 if phi_k > 1 else 3)
    sky_ref = float(np.median(R))
    return dict(R=(R - sky_ref).astype(np.float32), I=I.astype(np.float32), I_noiseless=I_nl,
                sigma_I=sig_i, phi_r=phi_r, phi_k=phi_k, snr=snr, snr_regime=snr_regime,
                sampling=samp, m=S10_M, seed=seed, sky_r=s_r, sky_i=s_i,
                R_noiseless=R_nl)


def s10_metrics(d: dict, theta, diff) -> dict:
    """Fit-quality metrics of the accuracy study (Sec. 3.3) for one fitted
    pair: P = sum K (Eq. 3), MSE of M against the noiseless target (the
    definition printed in Sec. 3.3) and against the noisy target (MSE_noisy:
    the quantity the paper's tabulated MSE values follow, about the mean pixel
    variance), and the mean and variance (MFB, MFV) of the normalised
    residuals (I - M)/sigma_I over the N_data valid pixels.  theta, diff: the
    fit's float64 theta and float32 difference image (valid region)."""
    m = d["m"]
    h = m // 2
    th = np.asarray(theta, np.float64)
    D = np.asarray(diff, np.float64)
    v = (slice(h, d["I"].shape[0] - h), slice(h, d["I"].shape[1] - h))
    I = d["I"][v].astype(np.float64)
    M = I - D
    eps = D / d["sigma_I"][v]
    mfb = float(eps.mean())
    return dict(P=float(th[:m * m].sum()), MSE=float(np.mean((M - d["I_noiseless"][v]) ** 2)),
                MSE_noisy=float(np.mean(D * D)),
                MFB=mfb, MFV=float(np.sum((eps - mfb) ** 2) / (eps.size - 1)))

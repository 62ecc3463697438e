"""Shared helpers of the GPU tests: seeded inputs and the two sides' loss specs."""
import numpy as np

import oracle
from paper_2104_13715_gb300 import synth

SPECS = {
    "gauss-fixed": dict(rho="gauss", noise="fixed", var=1.0),
    "gauss-ccd": dict(rho="gauss", noise="ccd", sigma0=6.0, gain=1.5, var_floor=1e-6),
    "gauss-emccd": dict(rho="gauss", noise="emccd", gain=25.8 / 300, excess=2.0, var_floor=1e-6),
    "huber-ccd": dict(rho="huber", noise="ccd", sigma0=5.0, gain=1.0, huber_c=1.345,
                      var_floor=1e-6),
    "huber-fixed": dict(rho="huber", noise="fixed", huber_c=1.345, var=1.0),
    "cauchy-fixed": dict(rho="cauchy", noise="fixed", var=1.0),
    "cauchy-emccd": dict(rho="cauchy", noise="emccd", gain=2.0, excess=2.0, var_floor=1e-6),
}


def ospec(d):
    keys = ("rho", "noise", "sigma0", "gain", "excess", "huber_c", "var", "var_floor")
    return oracle.LossSpec(**{k: d[k] for k in keys if k in d})


def field(H, W, m, seed, n_per_px=0.002, sky=100.0, sigma_k=1.2, scale=1.1, b0=30.0):
    spec = synth.PairSpec(size=(H, W), n_stars=max(3, int(n_per_px * H * W)), m=m,
                          fwhm_ref=2.0, kernel_sigma=sigma_k, scale=scale, b0=b0, sky=sky,
                          flux=(1e2, 1e5), read=5.0, gain=1.0)
    return synth.make_pair(spec, seed)


def theta_start(m, I, rng=None, jitter=0.0):
    """Box-car start (Sec. 2.9) with B0 = median(I); optional positive jitter
    so that the point is generic."""
    th = np.full(m * m + 1, 1.0 / (m * m))
    if rng is not None and jitter:
        th[:-1] *= 1.0 + jitter * rng.uniform(-1, 1, m * m)
    th[-1] = float(np.median(I))
    return th


def rel_inf(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))

"""Precision study of the accumulation of the per-pixel terms:
float32 pixel arithmetic with float64 accumulation against the pure-float32
accumulation form, on the high-dynamic-range recipe (fluxes 1e1-1e6, sky 2000,
m = 21, CCD negative log-likelihood), both against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2104_13715_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nat():
    from paper_2104_13715_gb300 import native
    yield native
    native.set_accumulation(native.ACCUM_FP64)


def _spec_keys(d):
    return {k: v for k, v in d["loss"].items()
            if k in ("rho", "noise", "sigma0", "gain", "excess", "huber_c", "var", "var_floor")}


def _grad(nat, d, th, mode):
    nat.set_accumulation(mode)
    try:
        up = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        L, g = nat.loss_grad(up(d["R"]), up(d["I"]), d["m"], torch.from_numpy(th),
                             nat.loss_spec(**_spec_keys(d)))
        return L.item(), g.cpu().numpy()
    finally:
        nat.set_accumulation(nat.ACCUM_FP64)


def test_float64_accumulation_meets_the_gradient_tolerance_and_float32_does_worse(nat):
    d = synth.workload("hdr2048_m21_nll", seed=3, size=1024)
    m = d["m"]
    th = np.full(m * m + 1, 1.0 / (m * m))
    th[:-1] *= 1.0 + 0.3 * np.random.default_rng(3).uniform(-1, 1, m * m)
    th[-1] = float(np.median(d["I"]))
    spec = oracle.LossSpec(**_spec_keys(d))
    Lo, go = oracle.loss_grad(d["R"], d["I"], m, th, spec)
    L64, g64 = _grad(nat, d, th, nat.ACCUM_FP64)
    L32, g32 = _grad(nat, d, th, nat.ACCUM_FP32)
    e64 = np.max(np.abs(g64 - go)) / np.max(np.abs(go))
    e32 = np.max(np.abs(g32 - go)) / np.max(np.abs(go))
    assert e64 <= 1e-5, e64
    assert abs(L64 - Lo) <= 1e-6 * abs(Lo)
    assert e32 > e64 and abs(L32 - Lo) > abs(L64 - Lo), (e32, e64)


def test_mode_switch_is_validated_and_restored(nat):
    with pytest.raises(nat.DiaError):
        nat.set_accumulation(7)
    assert nat.get_accumulation() == nat.ACCUM_FP64
    nat.set_accumulation(nat.ACCUM_FP32)
    assert nat.get_accumulation() == nat.ACCUM_FP32
    nat.set_accumulation(nat.ACCUM_FP64)
    assert nat.get_accumulation() == nat.ACCUM_FP64

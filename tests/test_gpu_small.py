"""Parity of the streaming small-kernel evaluation (m = 1, 3, 5) with the FP64
oracle, through dia_loss_grad and dia_fit.

The streaming form runs when the images are 16-byte aligned with a row pitch
that is a multiple of 16 bytes; tests use such pitches (padded views where the
width is ragged).  The tiled kernel gives the same sums in another order, so
a result that differs from the tiled one in its last bits shows the streaming
form ran.  Tolerances as for the tiled kernel: loss and gradient <= 1e-5
relative (max norm) at non-stationary theta."""
import numpy as np
import pytest
import torch

import oracle
from paper_2104_13715_gb300 import synth
from tests._helpers import SPECS, field, ospec, rel_inf, theta_start

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def nat():
    from paper_2104_13715_gb300 import native
    return native


def _pitched(a, ld, dtype):
    """Device copy of a 2-D array in a buffer of row pitch ld (>= width)."""
    H, W = a.shape
    buf = torch.zeros((H, ld), dtype=dtype, device="cuda")
    buf[:, :W] = torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)
    return buf[:, :W]


def _eval(nat, d, m, th, spec, mask=None, var=None, flat=None, ld=None, small=True):
    W = d["R"].shape[1]
    ld = ld or W
    t = lambda a, dt=torch.float32: None if a is None else _pitched(a, ld, dt)
    nat.set_small_kernel(small)
    try:
        L, g = nat.loss_grad(t(d["R"]), t(d["I"]), m, torch.from_numpy(th), nat.loss_spec(**spec),
                             mask=t(mask, torch.uint8), var=t(var), flat=t(flat))
        return L.item(), g.cpu().numpy()
    finally:
        nat.set_small_kernel(True)


@pytest.mark.parametrize("name", list(SPECS))
@pytest.mark.parametrize("m", [1, 3, 5])
def test_losses_with_mask_and_maps(nat, name, m):
    """Every loss x variance model with a 10% mask and a variance or flat map,
    on a ragged 203 x 261 image held with a 272-float pitch."""
    spec = SPECS[name]
    d = field(203, 261, m, seed=400 + m)
    rng = np.random.default_rng(17 + m)
    mask = (rng.random(d["R"].shape) > 0.1).astype(np.uint8)
    var = rng.uniform(50, 400, d["R"].shape).astype(np.float32) if spec["noise"] == "fixed" else None
    flat = rng.uniform(0.9, 1.1, d["R"].shape).astype(np.float32) if spec["noise"] != "fixed" else None
    th = theta_start(m, d["I"], rng, jitter=0.3)
    L, g = _eval(nat, d, m, th, spec, mask, var, flat, ld=272)
    Lo, go = oracle.loss_grad(d["R"], d["I"], m, th, ospec(spec), mask=mask, var=var, flat=flat)
    assert L == pytest.approx(Lo, rel=TOL)
    assert rel_inf(g, go) <= TOL


@pytest.mark.parametrize("m", [1, 3, 5])
@pytest.mark.parametrize("shape", [(70, 5131), (3001, 40), (9, 1500), (600, 600)])
def test_strip_splits_and_edges(nat, m, shape):
    """Wide (many column blocks, two-row strips), tall (one column block,
    long strips), short and square images; the streaming form differs from
    the tiled kernel in its last bits (another summation order) and both
    match the oracle."""
    H, W = shape
    if m > min(H, W):
        pytest.skip("kernel larger than the image")
    d = field(H, W, m, seed=H + W + m, n_per_px=0.004)
    rng = np.random.default_rng(m)
    th = theta_start(m, d["I"], rng, jitter=0.4)
    th[:-1] *= 1.5   # well away from the optimum (the 1e-5 test needs a gradient
    #                  that is not a small difference of large float32 terms)
    ld = (W + 15) // 16 * 16
    spec = SPECS["huber-ccd"]
    L, g = _eval(nat, d, m, th, spec, ld=ld)
    Lt, gt = _eval(nat, d, m, th, spec, ld=ld, small=False)
    Lo, go = oracle.loss_grad(d["R"], d["I"], m, th, ospec(spec))
    assert L == pytest.approx(Lo, rel=TOL) and Lt == pytest.approx(Lo, rel=TOL)
    assert rel_inf(g, go) <= TOL and rel_inf(gt, go) <= TOL
    if m > 1 or H * W > 4096:
        assert not (np.array_equal(g, gt) and L == Lt), "the streaming form did not run"


def test_unaligned_pitch_falls_back_to_the_tiled_kernel(nat):
    """A row pitch that is not a multiple of 4 floats: the tiled kernel runs
    (bitwise the tiled result) and matches the oracle."""
    m = 3
    d = field(100, 301, m, seed=5)
    th = theta_start(m, d["I"], np.random.default_rng(1), jitter=0.3)
    spec = SPECS["gauss-fixed"]
    L, g = _eval(nat, d, m, th, spec)
    Lt, gt = _eval(nat, d, m, th, spec, small=False)
    assert L == Lt and np.array_equal(g, gt)
    Lo, go = oracle.loss_grad(d["R"], d["I"], m, th, ospec(spec))
    assert rel_inf(g, go) <= TOL


def test_all_masked_gives_zero(nat):
    m = 5
    d = field(64, 128, m, seed=2)
    th = theta_start(m, d["I"])
    mask = np.zeros(d["R"].shape, np.uint8)
    L, g = _eval(nat, d, m, th, SPECS["gauss-ccd"], mask=mask)
    assert L == 0.0 and np.all(g == 0.0)


def test_bitwise_repeatable(nat):
    m = 5
    d = field(500, 512, m, seed=8)
    th = theta_start(m, d["I"], np.random.default_rng(2), jitter=0.2)
    a = _eval(nat, d, m, th, SPECS["huber-ccd"])
    b = _eval(nat, d, m, th, SPECS["huber-ccd"])
    assert a[0] == b[0] and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("name", ["ccd4096_m3_chi2", "ccd4096_m5_chi2"])
def test_full_size_workloads(nat, name):
    """The 4096^2 small-kernel workloads (the bench's memory-bound cases):
    loss and gradient at the box-car start and at a jittered point against
    the whole-image FP64 oracle."""
    d = synth.workload(name, seed=0)
    m = d["m"]
    spec = dict(rho="gauss", noise="fixed", var=1.0)
    rng = np.random.default_rng(3)
    for th in (theta_start(m, d["I"]), theta_start(m, d["I"], rng, jitter=0.5)):
        L, g = _eval(nat, d, m, th, spec)
        Lo, go = oracle.loss_grad(d["R"], d["I"], m, th, ospec(spec))
        assert L == pytest.approx(Lo, rel=TOL)
        assert rel_inf(g, go) <= TOL


def test_chi2_fit_matches_normal_equations(nat):
    """dia_fit at m = 5 (every optimiser iteration through the streaming
    form) against the B08 normal-equation solve."""
    m = 5
    d = field(384, 400, m, seed=21, sigma_k=0.7)
    R = torch.from_numpy(d["R"]).cuda()
    I = torch.from_numpy(d["I"]).cuda()
    out = nat.fit(R, I, m, nat.loss_spec(**SPECS["gauss-fixed"]))
    th = out["theta"].cpu().numpy()
    ref = oracle.normal_solve(d["R"], d["I"], m)
    ek = np.max(np.abs(th[:-1] - ref[:-1])) / abs(ref[:-1].sum())
    eb = abs(th[-1] - ref[-1]) / float(np.median(d["I"]))
    assert out["info"]["status"] == 0 and ek <= 1e-4 and eb <= 1e-4, (ek, eb, out["info"])


def test_ccd_fit_with_clipping_matches_newton(nat):
    """dia_fit at m = 3, CCD NLL, two clip passes (the working mask has the
    pair's 16-byte pitch, so the streaming form runs in every pass): the
    FP64 oracle's Newton optimum on the returned mask."""
    m = 3
    d = field(320, 336, m, seed=33, sigma_k=0.6)
    R = torch.from_numpy(d["R"]).cuda()
    I = torch.from_numpy(d["I"]).cuda()
    spec = SPECS["gauss-ccd"]
    out = nat.fit(R, I, m, nat.loss_spec(**spec), nat.default_opts(clip_passes=2),
                  want_mask=True)
    assert out["info"]["status"] == 0
    th = out["theta"].cpu().numpy()
    mk = out["mask"].cpu().numpy()
    ref = oracle.newton(d["R"], d["I"], m, th, ospec(spec), mask=mk)
    ek = np.max(np.abs(th[:-1] - ref[:-1])) / abs(ref[:-1].sum())
    eb = abs(th[-1] - ref[-1]) / float(np.median(d["I"]))
    assert ek <= 1e-4 and eb <= 1e-4, (ek, eb)

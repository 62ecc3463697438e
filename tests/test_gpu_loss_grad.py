"""Parity of the fused loss + gradient kernel (dia_loss_grad through the C ABI)
with the FP64 oracle, element by element, on seeded star fields.

Tolerance: gradients <= 1e-5 relative in the max norm at non-stationary
theta; the loss <= 1e-5 relative (float32 pixel arithmetic, float64 sums)."""
import numpy as np
import pytest
import torch

import oracle
from tests._helpers import SPECS, field, ospec, rel_inf, theta_start

pytestmark = pytest.mark.gpu
TOL_G = 1e-5
TOL_L = 1e-5


@pytest.fixture(scope="module")
def nat():
    from paper_2104_13715_gb300 import native
    return native


def _run(nat, d, m, th, spec, mask=None, var=None, flat=None):
    dev = torch.device("cuda")
    t = lambda a, dt=torch.float32: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(dev, dt)
    L, g = nat.loss_grad(t(d["R"]), t(d["I"]), m, torch.from_numpy(th), nat.loss_spec(**spec),
                         mask=t(mask, torch.uint8), var=t(var), flat=t(flat))
    return L.item(), g.cpu().numpy()


@pytest.mark.parametrize("m", [1, 3, 5, 7, 9, 11, 13, 15, 17, 19, 21, 23, 25, 27, 29, 31])
def test_every_kernel_side_gauss_fixed(nat, m):
    """All instantiated kernel sides; a ragged 2-3 tile image."""
    d = field(150, 301, m, seed=m)
    rng = np.random.default_rng(m)
    th = theta_start(m, d["I"], rng, jitter=0.5)
    L, g = _run(nat, d, m, th, SPECS["gauss-fixed"])
    Lo, go = oracle.loss_grad(d["R"], d["I"], m, th, ospec(SPECS["gauss-fixed"]))
    assert L == pytest.approx(Lo, rel=TOL_L)
    assert rel_inf(g, go) <= TOL_G


def test_every_tile_variant(nat):
    """Each tile variant of each kernel side gives the oracle's loss and gradient."""
    for m in range(1, 32, 2):
        nv = nat.kernel_variants(m)
        d = field(140, 270, m, seed=50 + m)
        th = theta_start(m, d["I"], np.random.default_rng(m), jitter=0.3)
        Lo, go = oracle.loss_grad(d["R"], d["I"], m, th, ospec(SPECS["huber-ccd"]))
        try:
            for v in range(nv):
                nat.select_kernel_variant(m, v)
                L, g = _run(nat, d, m, th, SPECS["huber-ccd"])
                assert L == pytest.approx(Lo, rel=TOL_L), (m, v)
                assert rel_inf(g, go) <= TOL_G, (m, v)
        finally:
            nat.select_kernel_variant(m, 0)


@pytest.mark.parametrize("name", list(SPECS))
@pytest.mark.parametrize("m", [5, 19, 25])
def test_losses_with_mask_and_maps(nat, name, m):
    spec = SPECS[name]
    d = field(203, 261, m, seed=100 + m)
    rng = np.random.default_rng(7 + m)
    mask = (rng.random(d["R"].shape) > 0.1).astype(np.uint8)
    var = rng.uniform(50, 400, d["R"].shape).astype(np.float32) if spec["noise"] == "fixed" else None
    flat = rng.uniform(0.9, 1.1, d["R"].shape).astype(np.float32) if spec["noise"] != "fixed" else None
    th = theta_start(m, d["I"], rng, jitter=0.3)
    L, g = _run(nat, d, m, th, spec, mask, var, flat)
    Lo, go = oracle.loss_grad(d["R"], d["I"], m, th, ospec(spec), mask=mask, var=var, flat=flat)
    assert L == pytest.approx(Lo, rel=TOL_L)
    assert rel_inf(g, go) <= TOL_G


def test_edge_shapes(nat):
    rng = np.random.default_rng(3)
    # kernel as large as the image: a 1 x 1 valid region; and m = 1
    for (H, W, m) in [(25, 25, 25), (31, 40, 31), (7, 300, 7), (300, 9, 9), (1, 1, 1), (2, 129, 1)]:
        R = rng.uniform(0, 100, (H, W)).astype(np.float32)
        I = rng.uniform(50, 150, (H, W)).astype(np.float32)
        d = dict(R=R, I=I)
        th = theta_start(m, I, rng, jitter=0.5)
        L, g = _run(nat, d, m, th, SPECS["gauss-fixed"])
        Lo, go = oracle.loss_grad(R, I, m, th, ospec(SPECS["gauss-fixed"]))
        assert L == pytest.approx(Lo, rel=TOL_L), (H, W, m)
        assert rel_inf(g, go) <= TOL_G, (H, W, m)


def test_all_masked_gives_zero(nat):
    d = field(64, 64, 5, seed=1)
    mask = np.zeros((64, 64), np.uint8)
    th = theta_start(5, d["I"])
    L, g = _run(nat, d, 5, th, SPECS["gauss-fixed"], mask=mask)
    assert L == 0.0 and np.all(g == 0.0)


def test_pitched_rows(nat):
    """Row pitch ld > W: the kernel must honour the pitch."""
    m = 11
    d = field(100, 150, m, seed=5)
    dev = torch.device("cuda")
    big = torch.zeros((100, 160), dtype=torch.float32, device=dev)
    bigI = torch.zeros((100, 160), dtype=torch.float32, device=dev)
    big[:, :150] = torch.from_numpy(d["R"]).to(dev)
    bigI[:, :150] = torch.from_numpy(d["I"]).to(dev)
    th = theta_start(m, d["I"], np.random.default_rng(0), 0.2)
    L, g = nat.loss_grad(big[:, :150], bigI[:, :150], m, torch.from_numpy(th),
                         nat.loss_spec(**SPECS["gauss-fixed"]))
    Lo, go = oracle.loss_grad(d["R"], d["I"], m, th, ospec(SPECS["gauss-fixed"]))
    assert L.item() == pytest.approx(Lo, rel=TOL_L)
    assert rel_inf(g.cpu().numpy(), go) <= TOL_G


def test_bitwise_repeatable(nat):
    d = field(300, 300, 15, seed=9)
    th = theta_start(15, d["I"], np.random.default_rng(1), 0.3)
    a = _run(nat, d, 15, th, SPECS["gauss-ccd"])
    b = _run(nat, d, 15, th, SPECS["gauss-ccd"])
    assert a[0] == b[0] and np.array_equal(a[1], b[1])


def test_diff_image(nat):
    m = 9
    d = field(120, 140, m, seed=4)
    th = theta_start(m, d["I"], np.random.default_rng(2), 0.4)
    dev = torch.device("cuda")
    D = nat.diff_image(torch.from_numpy(d["R"]).to(dev), torch.from_numpy(d["I"]).to(dev), m,
                       torch.from_numpy(th)).cpu().numpy()
    Do = oracle.diff_image(d["R"], d["I"], m, th)
    scale = np.max(np.abs(d["I"]))
    assert np.max(np.abs(D - Do)) <= 1e-6 * scale


def test_autograd_function_central_difference(nat):
    """DiaLossGrad (hand-written backward) vs a central difference of its own
    float32-pixel forward along the gradient direction, and vs the oracle."""
    m = 7
    d = field(96, 96, m, seed=11)
    dev = torch.device("cuda")
    R = torch.from_numpy(d["R"]).to(dev)
    I = torch.from_numpy(d["I"]).to(dev)
    spec = nat.loss_spec(**SPECS["gauss-ccd"])
    th = torch.tensor(theta_start(m, d["I"], np.random.default_rng(5), 0.3), device=dev,
                      requires_grad=True)
    L = nat.dia_loss(th, R, I, m, spec)
    L.backward()
    g = th.grad.detach().clone()
    v = g / g.norm()
    eps = 1e-3 * L.item() / float(g.norm())     # a 1e-3 relative change of the loss
    with torch.no_grad():
        Lp = nat.dia_loss(th + eps * v, R, I, m, spec)
        Lm = nat.dia_loss(th - eps * v, R, I, m, spec)
    fd = (Lp - Lm).item() / (2 * eps)
    assert fd == pytest.approx(float(g @ v), rel=1e-3)
    _, go = oracle.loss_grad(d["R"], d["I"], m, th.detach().cpu().numpy(), ospec(SPECS["gauss-ccd"]))
    assert rel_inf(g.cpu().numpy(), go) <= TOL_G


# (scalar variant, packed-float2 variant) of the same tile shape, from the
# VARIANTS table of paper_2104_13715_gb300/csrc/gen_instances.py
F2_TWINS = {25: [(2, 0), (1, 5), (3, 6)], 19: [(0, 3), (1, 4)], 11: [(2, 0)], 21: [(1, 0)],
            7: [(0, 2)], 9: [(1, 3), (4, 0)], 13: [(0, 3)], 15: [(1, 3)], 17: [(1, 2)], 23: [(1, 2)]}


@pytest.mark.parametrize("m", sorted(F2_TWINS))
def test_packed_fma_variants_are_bitwise_equal(nat, m):
    """__ffma2_rn performs the same correctly rounded FMAs in the same order as
    the scalar path, so the loss and gradient are identical bit for bit."""
    d = field(150, 260, m, seed=90 + m)
    th = theta_start(m, d["I"], np.random.default_rng(m), jitter=0.3)
    try:
        for a, b in F2_TWINS[m]:
            nat.select_kernel_variant(m, a)
            La, ga = _run(nat, d, m, th, SPECS["cauchy-emccd"])
            nat.select_kernel_variant(m, b)
            Lb, gb = _run(nat, d, m, th, SPECS["cauchy-emccd"])
            assert La == Lb and np.array_equal(ga, gb), (m, a, b)
    finally:
        nat.select_kernel_variant(m, 0)

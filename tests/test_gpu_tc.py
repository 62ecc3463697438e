"""Tensor-core forward (dia_diff_image_tc: tcgen05.mma on split-bf16 operands,
float32 accumulators in tensor memory) against the FP64 oracle's difference
image and the float32 CUDA-core form.

Tolerance, from the arithmetic: each operand x is carried as hi + lo with hi =
bf16(x) and lo = bf16(x - hi) (|x - hi - lo| <= 2^-17 |x|), and the product's
lo*lo term (<= 2^-16 |x y|) is dropped, so every term K R of M is off by at most
about 3 x 2^-16 |K R|: |D - D*| <= 2^-14 (|K| * |R|)_p + 1e-6 max |I| per pixel,
with (|K| * |R|) the correlation of the absolute values (the float32
accumulation adds far less)."""
import numpy as np
import pytest
import torch

import oracle
from tests._helpers import SPECS, field, ospec, rel_inf, theta_start

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nat():
    from paper_2104_13715_gb300 import native
    return native


def _t(a, dt=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)


def _bound(d, m, th):
    """2^-14 (|K| * |R|) + 1e-6 max |I| over the valid region."""
    ab = np.append(np.abs(th[:-1]), 0.0)
    return 2.0 ** -14 * oracle.model(np.abs(d["R"]), ab, m) + 1e-6 * np.max(np.abs(d["I"]))


@pytest.mark.parametrize("m", [1, 3, 7, 11, 19, 25, 31])
@pytest.mark.parametrize("shape", [(200, 300), (157, 131), (48, 64)])
def test_tc_difference_image_matches_the_oracle(nat, m, shape):
    d = field(shape[0], shape[1], m, seed=7 + m)
    rng = np.random.default_rng(m)
    th = np.append(np.abs(rng.normal(1.0 / (m * m), 0.3 / (m * m), m * m)), 97.5)
    D = nat.diff_image_tc(_t(d["R"]), _t(d["I"]), m, torch.from_numpy(th)).cpu().numpy()
    Do = oracle.diff_image(d["R"], d["I"], m, th)
    assert D.shape == Do.shape
    bound = _bound(d, m, th)
    assert np.all(np.abs(D - Do) <= bound), np.max(np.abs(D - Do) / bound)
    # and, where many taps average the split's rounding (m >= 7), a figure well
    # inside the bound (measured ~3e-7 of max |I| at 4096^2, m = 25); a lost
    # cross term of the split would exceed it
    if m >= 7:
        assert np.max(np.abs(D - Do)) <= 1e-5 * np.max(np.abs(d["I"]))
    Df = nat.diff_image(_t(d["R"]), _t(d["I"]), m, torch.from_numpy(th)).cpu().numpy()
    assert np.all(np.abs(D - Df) <= bound)


def test_tc_pitched_rows_and_signed_kernel(nat):
    """Row pitch > W and a kernel with negative taps (a difference of Gaussians)."""
    m, H, W, ld = 9, 140, 170, 192
    d = field(H, W, m, seed=5)
    Rp = np.zeros((H, ld), np.float32)
    Ip = np.zeros((H, ld), np.float32)
    Rp[:, :W] = d["R"]
    Ip[:, :W] = d["I"]
    yy, xx = np.mgrid[0:m, 0:m] - m // 2
    K = np.exp(-(xx ** 2 + yy ** 2) / 2.0) - 0.5 * np.exp(-(xx ** 2 + yy ** 2) / 8.0)
    th = np.append(K.ravel(), -12.0)
    R = _t(Rp)[:, :W]
    I = _t(Ip)[:, :W]
    D = nat.diff_image_tc(R, I, m, torch.from_numpy(th)).cpu().numpy()
    Do = oracle.diff_image(d["R"], d["I"], m, th)
    assert np.all(np.abs(D - Do) <= _bound(d, m, th))


def test_tc_rejects_polynomial_background(nat):
    import ctypes
    d = field(64, 64, 3, seed=1)
    R, I = _t(d["R"]), _t(d["I"])
    pair, keep = nat.make_pair(R, I, 3, bg_degree=1)
    th = torch.zeros(9 + 3, dtype=torch.float64, device="cuda")
    out = torch.empty((62, 62), dtype=torch.float32, device="cuda")
    ws = nat.workspace(64, 64, 3, device=R.device)
    st = nat.lib.dia_diff_image_tc(ctypes.byref(pair), ctypes.c_void_p(th.data_ptr()),
                                   ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(ws.data_ptr()),
                                   ws.numel(), None)
    assert st == nat.DIA_ERR_UNSUPPORTED


def test_tc_wait_timeout_aborts_cleanly(nat):
    """With a 300-cycle limit on the kernel's pipeline waits, the MMA role's
    first wait (for a window that has to come from memory) runs out: every
    role leaves (copies and MMAs in flight drained, tensor memory released)
    and the call returns DIA_ERR_TIMEOUT.  The next call, with the default
    limit, on the same stream and workspace gives the correct image."""
    import ctypes
    m = 11
    d = field(200, 300, m, seed=3)
    R, I = _t(d["R"]), _t(d["I"])
    th = torch.from_numpy(np.append(np.full(m * m, 1.0 / (m * m)), 90.0))
    pair, keep = nat.make_pair(R, I, m)
    ws = nat.workspace(200, 300, m, device=R.device)
    out = torch.empty((190, 290), dtype=torch.float32, device="cuda")
    thd = th.cuda()
    assert nat.lib.dia_set_tc_wait_cycles(-1) == nat.DIA_ERR_ARG
    assert nat.lib.dia_set_tc_wait_cycles(300) == 0
    try:
        st = nat.lib.dia_diff_image_tc(ctypes.byref(pair), ctypes.c_void_p(thd.data_ptr()),
                                       ctypes.c_void_p(out.data_ptr()),
                                       ctypes.c_void_p(ws.data_ptr()), ws.numel(), None)
    finally:
        assert nat.lib.dia_set_tc_wait_cycles(0) == 0
    assert st == nat.DIA_ERR_TIMEOUT
    torch.cuda.synchronize()
    D = nat.diff_image_tc(R, I, m, th, ws=ws).cpu().numpy()
    Do = oracle.diff_image(d["R"], d["I"], m, th.numpy())
    assert np.all(np.abs(D - Do) <= _bound(d, m, th.numpy()))


def _abscorr(Rabs, w, m):
    """sum_p w_p |R|[p + (a, b)] for every kernel pixel (a, b): the
    correlation of a valid-region weight map with |R|."""
    from numpy.lib.stride_tricks import sliding_window_view
    win = sliding_window_view(Rabs, (m, m))
    return np.einsum("yx,yxab->ab", w, win).ravel()


@pytest.mark.parametrize("m,name", [(3, "gauss-fixed"), (11, "gauss-ccd"), (19, "huber-fixed"),
                                    (25, "cauchy-fixed"), (31, "gauss-emccd")])
def test_tc_loss_grad_within_its_error_bound(nat, m, name):
    """dia_loss_grad_tc against the FP64 oracle within the bound its arithmetic
    gives: the forward pass's split-bf16 error |dM| <= 2^-14 (|K| * |R|)_p
    moves g_p by at most |l''(M_p)| |dM_p|; the float16 split of the weight
    gradient leaves ~2^-21 of each product (2^-19 taken); plus the float32
    floor 1e-6 max |grad|.  Per parameter k:
        |grad_k - grad*_k| <= sum_p |l''_p| |dM_p| |phi_k(p)| + 2^-19 sum_p |g_p| |phi_k(p)| + floor
    with phi_k the R window pixel of k (1 for B0)."""
    from tests._helpers import SPECS, ospec, theta_start
    spec = SPECS[name]
    d = field(200, 300, m, seed=60 + m)
    rng = np.random.default_rng(m)
    var = rng.uniform(50, 400, d["R"].shape).astype(np.float32) if spec["noise"] == "fixed" else None
    th = theta_start(m, d["I"], rng, jitter=0.3)
    L, g = nat.loss_grad_tc(_t(d["R"]), _t(d["I"]), m, torch.from_numpy(th), nat.loss_spec(**spec),
                            var=None if var is None else _t(var))
    g = g.cpu().numpy()
    Lo, go = oracle.loss_grad(d["R"], d["I"], m, th, ospec(spec), var=var)
    M = oracle.model(d["R"], th, m)
    _, g1, g2, _ = oracle.pixel_terms(d["I"], M, m, ospec(spec), var=var)
    dM = 2.0 ** -14 * oracle.model(np.abs(d["R"]), np.append(np.abs(th[:-1]), 0.0), m) + \
        1e-6 * np.max(np.abs(d["I"]))
    Rabs = np.abs(d["R"].astype(np.float64))
    wf = np.abs(g2) * dM
    bound = np.append(_abscorr(Rabs, wf, m), wf.sum())
    bound += 2.0 ** -19 * np.append(_abscorr(Rabs, np.abs(g1), m), np.abs(g1).sum())
    bound += 1e-6 * np.max(np.abs(go))
    assert np.all(np.abs(g - go) <= bound), np.max(np.abs(g - go) / bound)
    # the loss moves by at most sum_p |l'_p| |dM_p| (plus the float32 floor)
    assert abs(L.item() - Lo) <= np.sum(np.abs(g1) * dM) + 1e-6 * abs(Lo)


def test_tc_loss_grad_full_size_and_fp32_agree(nat):
    """4096^2, m = 25, Cauchy loss with mask and variance map (the headline
    workload) at the box-car start: the tensor-core evaluation's gradient is
    within 1e-5 of the FP64 oracle's (max norm)."""
    from paper_2104_13715_gb300 import synth
    from tests._helpers import rel_inf
    d = synth.workload("ccd4096_m25_cauchy_clip3", seed=0)
    m = d["m"]
    th = np.full(m * m + 1, 1.0 / (m * m))
    th[-1] = float(np.median(d["I"]))
    spec = dict(rho="cauchy", noise="fixed")
    L, g = nat.loss_grad_tc(_t(d["R"]), _t(d["I"]), m, torch.from_numpy(th), nat.loss_spec(**spec),
                            mask=_t(d["mask"], torch.uint8), var=_t(d["var"]))
    Lo, go = oracle.loss_grad(d["R"], d["I"], m, th, oracle.LossSpec(rho="cauchy", noise="fixed"),
                              mask=d["mask"], var=d["var"])
    assert rel_inf(g.cpu().numpy(), go) <= 1e-5
    assert L.item() == pytest.approx(Lo, rel=1e-5)


def test_tc_loss_grad_wait_timeout_aborts_cleanly(nat):
    """dia_loss_grad_tc with a 300-cycle wait limit: the forward pass's first
    waits run out and so do the weight-gradient kernel's (its MMA lane drains
    what it issued, the read-back pairs leave together); the call returns
    DIA_ERR_TIMEOUT.  With the default limit restored, the next call on the
    same tensors gives the oracle's gradient."""
    import ctypes
    m = 13
    d = field(300, 420, m, seed=31)
    spec = SPECS["gauss-ccd"]
    th = theta_start(m, d["I"], np.random.default_rng(3), jitter=0.2)
    R, I = _t(d["R"]), _t(d["I"])
    pair, keep = nat.make_pair(R, I, m)
    nb = nat.lib.dia_tc_workspace_size(pair.H, pair.W, pair.ld, m)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    thd = torch.from_numpy(th).cuda()
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    grad = torch.empty(m * m + 1, dtype=torch.float64, device="cuda")
    sp = nat.loss_spec(**spec)
    assert nat.lib.dia_set_tc_wait_cycles(300) == 0
    try:
        st = nat.lib.dia_loss_grad_tc(ctypes.byref(pair), ctypes.byref(sp),
                                      ctypes.c_void_p(thd.data_ptr()), ctypes.c_void_p(loss.data_ptr()),
                                      ctypes.c_void_p(grad.data_ptr()), ctypes.c_void_p(ws.data_ptr()),
                                      nb, None)
    finally:
        assert nat.lib.dia_set_tc_wait_cycles(0) == 0
    assert st == nat.DIA_ERR_TIMEOUT
    torch.cuda.synchronize()
    L, g = nat.loss_grad_tc(R, I, m, torch.from_numpy(th), sp)
    Lo, go = oracle.loss_grad(d["R"], d["I"], m, th, ospec(spec))
    assert rel_inf(g.cpu().numpy(), go) <= 1e-5


def test_tc_loss_grad_with_flat_field_and_mask(nat):
    """CCD variance with a flat field (v = s0^2 / F^2 + M / (G F)) and a mask
    through the tensor-core evaluation, against the oracle (1e-5 max norm)."""
    from tests._helpers import ospec, rel_inf, theta_start
    m = 21
    spec = SPECS["gauss-ccd"]
    d = field(280, 360, m, seed=44)
    rng = np.random.default_rng(5)
    flat = rng.uniform(0.85, 1.15, d["R"].shape).astype(np.float32)
    mask = (rng.random(d["R"].shape) > 0.07).astype(np.uint8)
    th = theta_start(m, d["I"], rng, jitter=0.3)
    L, g = nat.loss_grad_tc(_t(d["R"]), _t(d["I"]), m, torch.from_numpy(th), nat.loss_spec(**spec),
                            mask=_t(mask, torch.uint8), flat=_t(flat))
    Lo, go = oracle.loss_grad(d["R"], d["I"], m, th, ospec(spec), mask=mask, flat=flat)
    assert rel_inf(g.cpu().numpy(), go) <= 1e-5
    assert L.item() == pytest.approx(Lo, rel=1e-5)

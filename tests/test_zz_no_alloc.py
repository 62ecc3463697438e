"""dia_loss_grad_noalloc: the evaluation for callers that cannot allocate
device memory (for example code inside a host application whose device
memory is all owned by that application's pool, or a pipeline that must not
allocate once running).  It must give the same loss and gradient as
dia_loss_grad, which uses a caller workspace, on consecutive calls that share
the library's fixed scratch array.

This file is collected last on purpose: if it fails, a run stopping at the
first failure has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

from tests._helpers import SPECS, field, rel_inf, theta_start

pytestmark = pytest.mark.gpu
TOL = 1e-5   # the tolerance of the fused-kernel parity tests


@pytest.fixture(scope="module")
def nat():
    from paper_2104_13715_gb300 import native
    return native


@pytest.mark.parametrize("m,shape,name", [(25, (150, 301), "gauss-fixed"),
                                          (11, (203, 261), "gauss-ccd"),
                                          (31, (96, 420), "cauchy-fixed")])
def test_matches_workspace_entry_on_two_calls(nat, m, shape, name):
    d = field(*shape, m, seed=300 + m)
    dev = torch.device("cuda")
    R = torch.from_numpy(d["R"]).to(dev)
    I = torch.from_numpy(d["I"]).to(dev)
    spec = nat.loss_spec(**SPECS[name])
    rng = np.random.default_rng(m)
    mask = torch.from_numpy((rng.random(shape) > 0.05).astype(np.uint8)).to(dev)
    th1 = torch.from_numpy(theta_start(m, d["I"], rng, jitter=0.4))
    th2 = torch.from_numpy(theta_start(m, d["I"], rng, jitter=0.4))
    for th in (th1, th2):      # two calls in a row through the shared scratch array
        L0, g0 = nat.loss_grad(R, I, m, th, spec, mask=mask)
        L1, g1 = nat.loss_grad_noalloc(R, I, m, th, spec, mask=mask)
        torch.cuda.synchronize()
        assert L1.item() == pytest.approx(L0.item(), rel=TOL)
        assert rel_inf(g1.cpu().numpy(), g0.cpu().numpy()) <= TOL


def test_large_image_caps_the_grid_and_allocates_nothing(nat):
    """2048^2 at m = 31: about a thousand tiles against one resident CTA per
    SM, so every CTA loops over several tiles (the array's CTA cap, about 265
    at m = 31, is above the resident count on a 152-SM GPU).  Same result as
    dia_loss_grad on two calls in a row, and after a warm-up the call changes
    no device memory figure (free bytes from cudaMemGetInfo, torch's
    allocated bytes)."""
    m = 31
    d = field(2048, 2048, m, seed=77)
    dev = torch.device("cuda")
    R = torch.from_numpy(d["R"]).to(dev)
    I = torch.from_numpy(d["I"]).to(dev)
    spec = nat.loss_spec(**SPECS["cauchy-fixed"])
    rng = np.random.default_rng(9)
    th = torch.from_numpy(theta_start(m, d["I"], rng, jitter=0.4)).to(dev)
    pair, keep = nat.make_pair(R, I, m)
    n = m * m + 1
    out = torch.zeros(n + 1, dtype=torch.float64, device=dev)

    def call():
        return nat.lib.dia_loss_grad_noalloc(ctypes.byref(pair), ctypes.byref(spec),
                                             ctypes.c_void_p(th.data_ptr()),
                                             ctypes.c_void_p(out.data_ptr()),
                                             ctypes.c_void_p(out.data_ptr() + 8), None)

    L0, g0 = nat.loss_grad(R, I, m, th, spec)
    assert call() == 0          # warm-up: the first call on a device looks up the array
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(2):
        out.zero_()
        assert call() == 0
        torch.cuda.synchronize()
        assert out[0].item() == pytest.approx(L0.item(), rel=TOL)
        assert rel_inf(out[1:].cpu().numpy(), g0.cpu().numpy()) <= TOL
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0 and torch.cuda.memory_allocated() == alloc0


def test_rejects_unsupported_sizes(nat):
    dev = torch.device("cuda")
    R = torch.zeros((40, 40), device=dev)
    spec = nat.loss_spec()
    th = torch.zeros(33 * 33 + 1, dtype=torch.float64, device=dev)
    pair, _ = nat.make_pair(R, R, 33)
    out = torch.zeros(33 * 33 + 2, dtype=torch.float64, device=dev)
    st = nat.lib.dia_loss_grad_noalloc(ctypes.byref(pair), ctypes.byref(spec),
                                       ctypes.c_void_p(th.data_ptr()),
                                       ctypes.c_void_p(out.data_ptr()),
                                       ctypes.c_void_p(out.data_ptr() + 8), None)
    assert st == nat.DIA_ERR_UNSUPPORTED

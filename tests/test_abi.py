"""The C-ABI library loads and exports every entry point include/dia.h
declares; host-side argument checks need no GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dia.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dia_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def native():
    import __graft_entry__ as g
    from paper_2104_13715_gb300 import build
    build.build()
    from paper_2104_13715_gb300 import native
    return native


def test_every_declared_symbol_is_exported(native):
    names = _declared()
    assert "dia_fit" in names and "dia_loss_grad" in names
    lib = ctypes.CDLL(native.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    # and the binding wraps each of them
    assert set(names) <= set(native._SIGS)


def test_status_strings_and_version(native):
    assert native.status_str(0) == "DIA_OK"
    assert native.status_str(9) == "DIA_ERR_UNSUPPORTED"
    assert native.lib.dia_abi_version() == native.ABI_VERSION == 4


def test_default_opts_are_the_paper_values(native):
    o = native.default_opts()
    assert o.lr_kernel == 1e-3            # Sec. 2.9
    assert o.switch_tol == 1e-6           # Sec. 2.9
    assert o.clip_kappa == 5.0            # Sec. 4.2
    assert o.grad_tol == 1e-7             # Sec. 2.9
    # preconditioned L-BFGS settings (not in the paper; chosen by measurement)
    assert (o.precond, o.history, o.stall_iters, o.stall_iters_diag, o.max_ls_evals) == \
        (1, 20, 30, 1000, 12)


@pytest.mark.parametrize("H,W,ld,m,ok", [(128, 128, 128, 11, True), (10, 10, 10, 11, False),
                                         (64, 64, 60, 5, False), (64, 64, 64, 4, False),
                                         (64, 64, 64, 33, False), (33, 40, 48, 31, True),
                                         (1, 1, 1, 1, True)])
def test_workspace_size_validation(native, H, W, ld, m, ok):
    n = native.lib.dia_workspace_size(H, W, ld, m, 0, 0)
    assert (n > 0) == ok
    if ok:
        assert n % 256 == 0
        assert native.lib.dia_workspace_size(H, W, ld, m, 1, 1) > n


def test_arguments_rejected_before_any_launch(native):
    # NULL pair / bad kernel side: DIA_ERR_ARG without touching a GPU
    assert native.lib.dia_loss_grad(None, None, None, None, None, None, 0, None) == native.DIA_ERR_ARG
    p = native.Pair(1, 2, None, None, None, 16, 16, 16, 4, 0)      # even m
    spec = native.loss_spec()
    assert native.lib.dia_loss_grad(ctypes.byref(p), ctypes.byref(spec), 1, 1, 1, None, 0,
                                    None) == native.DIA_ERR_ARG
    p = native.Pair(1, 2, None, None, None, 40, 40, 40, 33, 0)     # m > DIA_MAX_M
    assert native.lib.dia_loss_grad(ctypes.byref(p), ctypes.byref(spec), 1, 1, 1, None, 0,
                                    None) == native.DIA_ERR_UNSUPPORTED
    bad = native.loss_spec(noise="ccd", gain=0.0)
    p = native.Pair(1, 2, None, None, None, 16, 16, 16, 3, 0)
    assert native.lib.dia_loss_grad(ctypes.byref(p), ctypes.byref(bad), 1, 1, 1, None, 0,
                                    None) == native.DIA_ERR_ARG
    # background degree outside [0, DIA_MAX_BG_DEGREE] (Eq. 18)
    for deg in (-1, 5):
        pd = native.Pair(1, 2, None, None, None, 16, 16, 16, 3, 0, deg)
        assert native.lib.dia_loss_grad(ctypes.byref(pd), ctypes.byref(spec), 1, 1, 1, 256,
                                        1 << 30, None) == native.DIA_ERR_ARG
        assert native.lib.dia_loss_grad_noalloc(ctypes.byref(pd), ctypes.byref(spec), 1, 1, 1,
                                                None) == native.DIA_ERR_ARG
    assert native.n_params(5, 0) == 26 and native.n_params(5, 2) == 31
    # workspace too small
    assert native.lib.dia_loss_grad(ctypes.byref(p), ctypes.byref(spec), 1, 1, 1, 256, 8,
                                    None) == native.DIA_ERR_WORKSPACE
    o = native.default_opts(history=0)
    assert native.lib.dia_fit(ctypes.byref(p), ctypes.byref(spec), ctypes.byref(o), None, None,
                              None, None, None, None, None, 0, None) == native.DIA_ERR_ARG


def test_model_extension_defaults_and_batch_validation(native):
    """The regulariser is off and the background constant by default (the
    paper's fits, Sec. 3.3, use neither); the batch planner sizes each pair's
    theta as m*m + (d+1)(d+2)/2 and rejects a degree outside [0, 4] before
    anything runs (host-only calls)."""
    o = native.default_opts()
    assert o.reg_lambda == 0.0
    pair = native.Pair(1, 2, None, None, None, 64, 64, 64, 5, 0)
    assert pair.bg_degree == 0
    pairs = (native.Pair * 2)(native.Pair(1, 2, None, None, None, 64, 64, 64, 5, 0, 0),
                              native.Pair(1, 2, None, None, None, 80, 72, 72, 7, 0, 2))
    n_ok = native.lib.dia_batch_workspace_size(pairs, 2, ctypes.byref(o))
    assert n_ok > 0
    pairs[1].bg_degree = 4
    assert native.lib.dia_batch_workspace_size(pairs, 2, ctypes.byref(o)) >= n_ok
    pairs[1].bg_degree = 5
    assert native.lib.dia_batch_workspace_size(pairs, 2, ctypes.byref(o)) == 0
    pairs[1].bg_degree = -1
    assert native.lib.dia_batch_workspace_size(pairs, 2, ctypes.byref(o)) == 0


def test_batch_entry_validates_before_launching(native):
    """dia_fit_batch: no pairs, a bad loss for one pair, or clipping requested
    give status codes without any device work (host-only)."""
    spec = native.loss_spec()
    o = native.default_opts()
    assert native.lib.dia_fit_batch(None, 2, ctypes.byref(spec), ctypes.byref(o), None, None,
                                    None, None, 0, None) == native.DIA_ERR_ARG
    pairs = (native.Pair * 2)(native.Pair(1, 2, None, None, None, 64, 64, 64, 5, 0),
                              native.Pair(1, 2, None, None, None, 64, 64, 64, 5, 0))
    bad = native.loss_spec(noise="ccd", gain=0.0)
    assert native.lib.dia_fit_batch(pairs, 2, ctypes.byref(bad), ctypes.byref(o), None, None,
                                    None, None, 0, None) == native.DIA_ERR_ARG
    clip = native.default_opts(clip_passes=1)
    assert native.lib.dia_fit_batch(pairs, 2, ctypes.byref(spec), ctypes.byref(clip), None, None,
                                    None, None, 0, None) == native.DIA_ERR_UNSUPPORTED
    big = (native.Pair * 1)(native.Pair(1, 2, None, None, None, 64, 64, 64, 33, 0))
    assert native.lib.dia_fit_batch(big, 1, ctypes.byref(spec), ctypes.byref(o), None, None,
                                    None, None, 0, None) == native.DIA_ERR_UNSUPPORTED


@pytest.mark.parametrize("field,value", [("history", 0), ("history", 129), ("graph_iters", 0),
                                         ("max_ls_evals", 1), ("timeout_s", 0.0),
                                         ("reg_lambda", -1.0), ("reg_lambda", float("nan")),
                                         ("init", 3), ("init", 2), ("clip_passes", -1),
                                         ("precond_window", -5), ("beta1", 1.0),
                                         ("beta1", -0.1), ("beta2", 1.0),
                                         ("lr_kernel", 0.0), ("lr_b0", -1.0),
                                         ("lr_kernel", float("inf")), ("adam_eps", 0.0),
                                         ("grad_tol", float("nan")), ("switch_tol", -1.0),
                                         ("rel_tol", float("inf"))])
def test_out_of_range_options_are_rejected_on_the_host(native, field, value):
    """Every entry validates dia_opts before any launch (init 2 without theta0
    included); the batch entry takes no theta0, so init 2 is refused there too."""
    spec = native.loss_spec()
    p = native.Pair(1, 2, None, None, None, 64, 64, 64, 5, 0)
    o = native.default_opts()
    setattr(o, field, value)
    assert native.lib.dia_fit(ctypes.byref(p), ctypes.byref(spec), ctypes.byref(o), None, None,
                              None, None, None, None, None, 0, None) == native.DIA_ERR_ARG
    pairs = (native.Pair * 1)(p)
    assert native.lib.dia_fit_batch(pairs, 1, ctypes.byref(spec), ctypes.byref(o), None, None,
                                    None, None, 0, None) == native.DIA_ERR_ARG


@pytest.mark.parametrize("kappa", [0.0, -1.0, float("nan"), float("inf")])
def test_clip_threshold_is_checked_when_clipping(native, kappa):
    """A clip threshold that is not positive and finite is refused when the fit
    clips (NaN would clip nothing, 0 every pixel); without clipping it is unused."""
    spec = native.loss_spec()
    p = native.Pair(1, 2, None, None, None, 64, 64, 64, 5, 0)
    o = native.default_opts(clip_passes=2)
    o.clip_kappa = kappa
    assert native.lib.dia_fit(ctypes.byref(p), ctypes.byref(spec), ctypes.byref(o), None, None,
                              None, None, None, None, None, 0, None) == native.DIA_ERR_ARG


def test_eval_form_switch_and_workspace_growth(native):
    """dia_set_eval_form takes DIA_EVAL_FP32 / DIA_EVAL_TC only; while the
    tensor-core form is set, the workspace of a pair it serves (m <= 31,
    constant background, one kernel) grows by at least the padded g map and
    keeps its size for m = 33 and for a polynomial background."""
    import torch
    assert native.lib.dia_set_eval_form(-1) == native.DIA_ERR_ARG
    assert native.lib.dia_set_eval_form(3) == native.DIA_ERR_ARG
    assert native.get_eval_form() == native.EVAL_FP32
    H, W = 1000, 1100
    base = native.lib.dia_workspace_size(H, W, W, 25, 0, 0)
    base33 = native.lib.dia_workspace_size(H, W, W, 33, 0, 0)
    R = torch.zeros((H, W))
    p_bg, _ = native.make_pair(R, R, 25, bg_degree=1)
    base_bg = native.lib.dia_pair_workspace_size(ctypes.byref(p_bg), 0)
    native.set_eval_form(native.EVAL_TC)
    try:
        assert native.get_eval_form() == native.EVAL_TC
        # 976 x 1076 valid pixels padded to 1024 x 1152
        assert native.lib.dia_workspace_size(H, W, W, 25, 0, 0) >= base + 1024 * 1152 * 4
        assert native.lib.dia_workspace_size(H, W, W, 33, 0, 0) == base33
        assert native.lib.dia_pair_workspace_size(ctypes.byref(p_bg), 0) == base_bg
    finally:
        native.set_eval_form(native.EVAL_FP32)
    assert native.lib.dia_workspace_size(H, W, W, 25, 0, 0) == base


def test_error_site_is_zero_before_any_cuda_error(native):
    """dia_last_cuda_error_site names the library line that caught the last
    CUDA error of this host thread, 0 while there has been none."""
    assert native.lib.dia_last_cuda_error() == 0
    assert native.lib.dia_last_cuda_error_site() == 0


def test_auto_eval_form_takes_the_tensor_cores_from_m_19(native):
    """DIA_EVAL_AUTO sizes the tensor-core regions only for 19 <= m <= 31."""
    H, W = 600, 640
    base = {m: native.lib.dia_workspace_size(H, W, W, m, 0, 0) for m in (15, 17, 19, 31)}
    native.set_eval_form(native.EVAL_AUTO)
    try:
        assert native.lib.dia_workspace_size(H, W, W, 15, 0, 0) == base[15]
        assert native.lib.dia_workspace_size(H, W, W, 17, 0, 0) == base[17]
        assert native.lib.dia_workspace_size(H, W, W, 19, 0, 0) > base[19]
        assert native.lib.dia_workspace_size(H, W, W, 31, 0, 0) > base[31]
    finally:
        native.set_eval_form(native.EVAL_FP32)


def test_batch_eval_timing_arguments(native):
    """dia_set_batch_eval_timing takes 0..1000 repetitions and
    dia_get_batch_eval_timing needs both output arrays (host-only calls)."""
    lib = native.lib
    assert lib.dia_set_batch_eval_timing(-1) == native.DIA_ERR_ARG
    assert lib.dia_set_batch_eval_timing(1001) == native.DIA_ERR_ARG
    assert lib.dia_set_batch_eval_timing(3) == native.DIA_OK
    assert lib.dia_set_batch_eval_timing(0) == native.DIA_OK
    ms = (ctypes.c_float * 4)()
    fl = (ctypes.c_double * 4)()
    assert lib.dia_get_batch_eval_timing(None, fl) == native.DIA_ERR_ARG
    assert lib.dia_get_batch_eval_timing(ms, None) == native.DIA_ERR_ARG
    assert lib.dia_get_batch_eval_timing(ms, fl) == native.DIA_OK

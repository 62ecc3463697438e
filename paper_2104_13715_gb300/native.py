"""ctypes binding of the C ABI in ``include/dia.h`` (argument marshalling only).

Every function here forwards to the CUDA library ``_dia_cuda.so``; there is no
CPU path.  If the library is missing the import of this module raises.  PyTorch
supplies device memory (images, outputs, the workspace) and the stream.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_dia_cuda.so")

DIA_OK, DIA_ERR_ARG, DIA_ERR_CUDA, DIA_ERR_NONFINITE, DIA_ERR_MAXITER = 0, 1, 2, 3, 4
DIA_ERR_LINESEARCH, DIA_ERR_DEGENERATE, DIA_ERR_TIMEOUT, DIA_ERR_WORKSPACE = 5, 6, 7, 8
DIA_ERR_UNSUPPORTED = 9
DIA_MAX_M = 31
RHO = {"gauss": 0, "huber": 1, "cauchy": 2}
VAR = {"fixed": 0, "ccd": 1, "emccd": 2}
MEM_DEVICE, MEM_HOST = 0, 1


class LossSpec(ctypes.Structure):
    _fields_ = [("rho", ctypes.c_int32), ("var_model", ctypes.c_int32),
                ("sigma0", ctypes.c_float), ("gain", ctypes.c_float),
                ("excess", ctypes.c_float), ("huber_c", ctypes.c_float),
                ("var_scalar", ctypes.c_float), ("var_floor", ctypes.c_float)]


class Pair(ctypes.Structure):
    _fields_ = [("ref", ctypes.c_void_p), ("img", ctypes.c_void_p), ("mask", ctypes.c_void_p),
                ("var", ctypes.c_void_p), ("flat", ctypes.c_void_p),
                ("H", ctypes.c_int32), ("W", ctypes.c_int32), ("ld", ctypes.c_int32),
                ("m", ctypes.c_int32), ("mem", ctypes.c_int32), ("bg_degree", ctypes.c_int32),
                ("kernel_degree", ctypes.c_int32)]


class Opts(ctypes.Structure):
    _fields_ = [("lr_kernel", ctypes.c_double), ("lr_b0", ctypes.c_double),
                ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("adam_eps", ctypes.c_double), ("switch_tol", ctypes.c_double),
                ("max_adam_iters", ctypes.c_int32), ("history", ctypes.c_int32),
                ("rel_tol", ctypes.c_double), ("grad_tol", ctypes.c_double),
                ("max_lbfgs_iters", ctypes.c_int32), ("max_evals", ctypes.c_int32),
                ("clip_passes", ctypes.c_int32), ("clip_kappa", ctypes.c_float),
                ("init", ctypes.c_int32), ("init_sigma", ctypes.c_double),
                ("theta0", ctypes.c_void_p), ("graph_iters", ctypes.c_int32),
                ("timeout_s", ctypes.c_double), ("stall_iters", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("precond", ctypes.c_int32),
                ("stall_iters_diag", ctypes.c_int32), ("max_ls_evals", ctypes.c_int32),
                ("precond_window", ctypes.c_int32), ("reg_lambda", ctypes.c_double)]


class FisherInfo(ctypes.Structure):
    _fields_ = [("positive_definite", ctypes.c_int32), ("n", ctypes.c_int32),
                ("log_det", ctypes.c_double), ("min_pivot", ctypes.c_double),
                ("ndata", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class FitInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("adam_iters", ctypes.c_int32),
                ("lbfgs_iters", ctypes.c_int32), ("evals", ctypes.c_int32),
                ("clip_passes_done", ctypes.c_int32), ("ndata", ctypes.c_int64),
                ("loss", ctypes.c_double), ("grad_inf", ctypes.c_double),
                ("scale", ctypes.c_double), ("b0", ctypes.c_double),
                ("reason", ctypes.c_int32), ("kernel_launches", ctypes.c_int64),
                ("precond_used", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# Every symbol include/dia.h declares, with its ctypes signature.
_P = ctypes.POINTER
_SIGS = {
    "dia_status_str": (ctypes.c_char_p, [ctypes.c_int32]),
    "dia_abi_version": (ctypes.c_int32, []),
    "dia_last_cuda_error": (ctypes.c_int32, []),
    "dia_last_cuda_error_site": (ctypes.c_int32, []),
    "dia_opts_default": (ctypes.c_int32, [_P(Opts)]),
    "dia_workspace_size": (ctypes.c_size_t, [ctypes.c_int32] * 6),
    "dia_kernel_variants": (ctypes.c_int32, [ctypes.c_int32]),
    "dia_select_kernel_variant": (ctypes.c_int32, [ctypes.c_int32, ctypes.c_int32]),
    "dia_kernel_variant_desc": (ctypes.c_int32, [ctypes.c_int32, ctypes.c_int32]
                                + [_P(ctypes.c_int32)] * 4),
    "dia_loss_grad": (ctypes.c_int32, [_P(Pair), _P(LossSpec), ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                       ctypes.c_void_p]),
    "dia_diff_image": (ctypes.c_int32, [_P(Pair), ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "dia_diff_image_tc": (ctypes.c_int32, [_P(Pair), ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "dia_loss_grad_noalloc": (ctypes.c_int32, [_P(Pair), _P(LossSpec), ctypes.c_void_p,
                                               ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_void_p]),
    "dia_batch_workspace_size": (ctypes.c_size_t, [_P(Pair), ctypes.c_int32, _P(Opts)]),
    "dia_fisher_workspace_size": (ctypes.c_size_t, [ctypes.c_int32] * 4),
    "dia_set_accumulation": (ctypes.c_int32, [ctypes.c_int32]),
    "dia_set_small_kernel": (ctypes.c_int32, [ctypes.c_int32]),
    "dia_select_batch_variant": (ctypes.c_int32, [ctypes.c_int32, ctypes.c_int32]),
    "dia_get_batch_variant": (ctypes.c_int32, [ctypes.c_int32]),
    "dia_set_batch_eval_timing": (ctypes.c_int32, [ctypes.c_int32]),
    "dia_get_batch_eval_timing": (ctypes.c_int32, [ctypes.POINTER(ctypes.c_float),
                                                   ctypes.POINTER(ctypes.c_double)]),
    "dia_batch_chunk_tiles": (ctypes.c_int32, [ctypes.c_int32, ctypes.c_int32]),
    "dia_set_tc_wait_cycles": (ctypes.c_int32, [ctypes.c_int64]),
    "dia_tc_workspace_size": (ctypes.c_size_t, [ctypes.c_int32] * 4),
    "dia_loss_grad_tc": (ctypes.c_int32, [_P(Pair), _P(LossSpec), ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                          ctypes.c_void_p]),
    "dia_pair_workspace_size": (ctypes.c_size_t, [_P(Pair), ctypes.c_int32]),
    "dia_pair_fisher_workspace_size": (ctypes.c_size_t, [_P(Pair)]),
    "dia_time_eval": (ctypes.c_int32, [_P(Pair), _P(LossSpec), ctypes.c_void_p, ctypes.c_int32,
                                       ctypes.c_void_p, ctypes.c_size_t,
                                       ctypes.POINTER(ctypes.c_float), ctypes.c_void_p,
                                       ctypes.c_size_t, ctypes.c_void_p]),
    "dia_get_small_kernel": (ctypes.c_int32, []),
    "dia_get_accumulation": (ctypes.c_int32, []),
    "dia_set_eval_form": (ctypes.c_int32, [ctypes.c_int32]),
    "dia_get_eval_form": (ctypes.c_int32, []),
    "dia_fisher": (ctypes.c_int32, [_P(Pair), _P(LossSpec), ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, _P(FisherInfo), ctypes.c_void_p,
                                    ctypes.c_size_t, ctypes.c_void_p]),
    "dia_fit_batch": (ctypes.c_int32, [_P(Pair), ctypes.c_int32, _P(LossSpec), _P(Opts),
                                       ctypes.c_void_p, ctypes.c_void_p, _P(FitInfo),
                                       ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "dia_fit": (ctypes.c_int32, [_P(Pair), _P(LossSpec), _P(Opts), ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_void_p, _P(FitInfo), ctypes.c_void_p, ctypes.c_size_t,
                                 ctypes.c_void_p]),
}


ABI_VERSION = 4   # the struct layouts below match include/dia.h of this version


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"CUDA library {LIB_PATH} is missing: run __graft_entry__.build() "
            "(there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if lib.dia_abi_version() != ABI_VERSION:
        raise ImportError(f"{LIB_PATH} has ABI version {lib.dia_abi_version()}, this binding "
                          f"expects {ABI_VERSION}: rebuild it with __graft_entry__.build()")
    return lib


lib = _load()


class DiaError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        name = lib.dia_status_str(status).decode()
        extra = (f" (cuda error {lib.dia_last_cuda_error()} at site {lib.dia_last_cuda_error_site()})"
                 if status == DIA_ERR_CUDA else "")
        super().__init__(f"{what}: {name}{extra}")


def _check(status, what):
    if status != DIA_OK:
        raise DiaError(status, what)


def status_str(s: int) -> str:
    return lib.dia_status_str(s).decode()


ACCUM_FP64, ACCUM_FP32 = 0, 1


def set_accumulation(mode: int) -> None:
    """dia_set_accumulation: ACCUM_FP64 (default) or ACCUM_FP32 (comparison form)."""
    _check(lib.dia_set_accumulation(int(mode)), "dia_set_accumulation")


EVAL_FP32, EVAL_TC, EVAL_AUTO = 0, 1, 2


def set_eval_form(form: int) -> None:
    """dia_set_eval_form: EVAL_FP32 (default, fused float32 kernels), EVAL_TC
    (both contractions on the tensor cores where they apply) or EVAL_AUTO (the
    tensor cores where they were measured faster: 19 <= m <= 31).  Size any
    workspace after choosing the form."""
    _check(lib.dia_set_eval_form(int(form)), "dia_set_eval_form")


def get_eval_form() -> int:
    return int(lib.dia_get_eval_form())


def set_small_kernel(enable: bool) -> None:
    """dia_set_small_kernel: the streaming small-kernel evaluation (m <= 5)
    on (default) or off (the tiled kernel for every m)."""
    _check(lib.dia_set_small_kernel(1 if enable else 0), "dia_set_small_kernel")


def set_batch_eval_timing(reps: int) -> None:
    """dia_set_batch_eval_timing: kernel-level timing of each group's batched
    evaluation kernel inside later fit_batch calls (0: off)."""
    _check(lib.dia_set_batch_eval_timing(int(reps)), "dia_set_batch_eval_timing")


def batch_eval_timing() -> dict:
    """dia_get_batch_eval_timing: per kernel-side group (0..3) the mean ms per
    launch and the algorithmic flop of the last timed fit_batch call."""
    ms = (ctypes.c_float * 4)()
    fl = (ctypes.c_double * 4)()
    _check(lib.dia_get_batch_eval_timing(ms, fl), "dia_get_batch_eval_timing")
    return {"ms": [float(x) for x in ms], "flop": [float(x) for x in fl]}


def select_batch_variant(group: int, variant: int) -> None:
    """dia_select_batch_variant: work-item size variant of a kernel-side group."""
    _check(lib.dia_select_batch_variant(group, variant), "dia_select_batch_variant")


def get_small_kernel() -> bool:
    return bool(lib.dia_get_small_kernel())


def get_accumulation() -> int:
    return lib.dia_get_accumulation()


def kernel_variants(m: int) -> int:
    return lib.dia_kernel_variants(m)


def select_kernel_variant(m: int, variant: int) -> None:
    _check(lib.dia_select_kernel_variant(m, variant), "dia_select_kernel_variant")


def kernel_variant_desc(m: int, variant: int = -1) -> dict:
    v = [ctypes.c_int32() for _ in range(4)]
    _check(lib.dia_kernel_variant_desc(m, variant, *[ctypes.byref(x) for x in v]),
           "dia_kernel_variant_desc")
    return dict(zip(("warps", "rows_per_warp", "tile_rows", "smem_bytes"), (x.value for x in v)))


def loss_spec(rho="gauss", noise="fixed", sigma0=0.0, gain=1.0, excess=2.0, huber_c=1.345,
              var=1.0, var_floor=1e-6, **_ignored) -> LossSpec:
    """dia_loss_spec from the plain loss keys shared with the oracle."""
    return LossSpec(RHO[rho], VAR[noise], sigma0, gain, excess, huber_c, var, var_floor)


def default_opts(**kw) -> Opts:
    o = Opts()
    _check(lib.dia_opts_default(ctypes.byref(o)), "dia_opts_default")
    for k, v in kw.items():
        if k == "theta0":
            raise ValueError("pass theta0 to fit()")
        setattr(o, k, v)
    return o


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _img(t, H, W, name, dtype=torch.float32):
    if t is None:
        return None
    if t.dtype != dtype or t.dim() != 2 or tuple(t.shape) != (H, W) or t.stride(1) != 1:
        raise ValueError(f"{name}: expected a row-major {dtype} tensor of shape {(H, W)}")
    return t


def n_params(m, bg_degree=0, kernel_degree=0):
    """Entries of theta: (dk+1)(dk+2)/2 kernels of m*m pixels (one unless the
    kernel varies over the image with degree dk) and (d+1)(d+2)/2 background
    coefficients (Eq. 18; 1 = the constant B0)."""
    return (kernel_degree + 1) * (kernel_degree + 2) // 2 * m * m + \
        (bg_degree + 1) * (bg_degree + 2) // 2


def make_pair(R, I, m, mask=None, var=None, flat=None, bg_degree=0, kernel_degree=0):
    """dia_pair over torch tensors (all on one CUDA device, or all on the host
    in pinned or pageable memory).  Returns (pair, keep-alive list)."""
    H, W = R.shape
    ld = R.stride(0)
    host = not R.is_cuda
    for name, t in (("I", I), ("mask", mask), ("var", var), ("flat", flat)):
        if t is not None:
            if t.is_cuda == host:
                raise ValueError(f"{name} must live where R lives")
            if t.stride(0) != ld:
                raise ValueError(f"{name} must share R's row pitch")
    _img(R, H, W, "R")
    _img(I, H, W, "I")
    _img(mask, H, W, "mask", torch.uint8)
    _img(var, H, W, "var")
    _img(flat, H, W, "flat")
    p = Pair(R.data_ptr(), I.data_ptr(), mask.data_ptr() if mask is not None else None,
             var.data_ptr() if var is not None else None,
             flat.data_ptr() if flat is not None else None, H, W, ld, m,
             MEM_HOST if host else MEM_DEVICE, bg_degree, kernel_degree)
    return p, [R, I, mask, var, flat]


def workspace_size(H, W, m, ld=None, clip=False, host=False) -> int:
    n = lib.dia_workspace_size(H, W, ld or W, m, int(bool(clip)), MEM_HOST if host else MEM_DEVICE)
    if n == 0:
        raise DiaError(DIA_ERR_ARG, "dia_workspace_size")
    return n


def workspace(H, W, m, ld=None, clip=False, host=False, device=None) -> torch.Tensor:
    """A device workspace tensor (256-byte aligned by the caching allocator)."""
    n = workspace_size(H, W, m, ld, clip, host)
    return torch.empty(n, dtype=torch.uint8, device=device or "cuda")


def pair_workspace(pair, clip=False, device=None) -> torch.Tensor:
    """Workspace for this dia_pair (dia_pair_workspace_size: any kernel degree)."""
    n = lib.dia_pair_workspace_size(ctypes.byref(pair), int(bool(clip)))
    if n == 0:
        raise DiaError(DIA_ERR_ARG, "dia_pair_workspace_size")
    return torch.empty(n, dtype=torch.uint8, device=device or "cuda")


def loss_grad(R, I, m, theta, spec: LossSpec, mask=None, var=None, flat=None, ws=None,
              stream=None, bg_degree=0, kernel_degree=0):
    """One fused evaluation on the device: returns (loss[1], grad[n]) float64 tensors.
    ``kernel_degree`` > 0: a spatially varying kernel of that degree."""
    pair, keep = make_pair(R, I, m, mask, var, flat, bg_degree, kernel_degree)
    if not R.is_cuda:
        raise ValueError("loss_grad takes device tensors")
    theta = theta.to(device=R.device, dtype=torch.float64).contiguous()
    n = n_params(m, bg_degree, kernel_degree)
    if theta.numel() != n:
        raise ValueError(f"theta must have {n} entries")
    ws = ws if ws is not None else pair_workspace(pair, device=R.device)
    loss = torch.empty(1, dtype=torch.float64, device=R.device)
    grad = torch.empty(n, dtype=torch.float64, device=R.device)
    st = lib.dia_loss_grad(ctypes.byref(pair), ctypes.byref(spec), _ptr(theta), _ptr(loss),
                           _ptr(grad), _ptr(ws), ws.numel(), _stream(stream))
    _check(st, "dia_loss_grad")
    return loss, grad


def time_eval(R, I, m, theta, spec: LossSpec, mask=None, var=None, flat=None, reps=20,
              flush=None, ws=None, stream=None, bg_degree=0) -> float:
    """dia_time_eval: mean device milliseconds of the fused evaluation kernel
    alone over `reps` launches (CUDA events on the stream), each after
    reading the uint8 device tensor `flush` (if given) through L2 to evict it;
    without `flush`, the launches run back to back between one pair of events."""
    pair, keep = make_pair(R, I, m, mask, var, flat, bg_degree)
    theta = theta.to(device=R.device, dtype=torch.float64).contiguous()
    ws = ws if ws is not None else workspace(pair.H, pair.W, m, pair.ld, device=R.device)
    ms = ctypes.c_float(0.0)
    st = lib.dia_time_eval(ctypes.byref(pair), ctypes.byref(spec), _ptr(theta), int(reps),
                           _ptr(flush), 0 if flush is None else flush.numel(), ctypes.byref(ms),
                           _ptr(ws), ws.numel(), _stream(stream))
    _check(st, "dia_time_eval")
    return float(ms.value)


def fisher(R, I, m, theta, spec: LossSpec, mask=None, var=None, flat=None, want_F=True,
           want_cov=True, stream=None, bg_degree=0, kernel_degree=0):
    """dia_fisher: observed Fisher information F (the Hessian of the loss at
    theta, Sec. 2.5) and the covariance estimate F^-1.  Returns dict(F, cov,
    info) with n x n float64 device tensors (None where not asked for; cov is
    NaN when F is not positive definite)."""
    pair, keep = make_pair(R, I, m, mask, var, flat, bg_degree, kernel_degree)
    if not R.is_cuda:
        raise ValueError("fisher takes device tensors")
    n = n_params(m, bg_degree, kernel_degree)
    theta = theta.to(device=R.device, dtype=torch.float64).contiguous()
    nb = lib.dia_pair_fisher_workspace_size(ctypes.byref(pair))
    if nb == 0:
        raise DiaError(DIA_ERR_ARG, "dia_fisher_workspace_size")
    ws = torch.empty(nb, dtype=torch.uint8, device=R.device)
    F = torch.empty((n, n), dtype=torch.float64, device=R.device) if want_F else None
    cov = torch.empty((n, n), dtype=torch.float64, device=R.device) if want_cov else None
    info = FisherInfo()
    st = lib.dia_fisher(ctypes.byref(pair), ctypes.byref(spec), _ptr(theta), _ptr(F), _ptr(cov),
                        ctypes.byref(info), _ptr(ws), nb, _stream(stream))
    _check(st, "dia_fisher")
    return {"F": F, "cov": cov, "info": info.as_dict()}


def loss_grad_noalloc(R, I, m, theta, spec: LossSpec, mask=None, var=None, flat=None,
                      stream=None, bg_degree=0):
    """dia_loss_grad_noalloc: the same evaluation without a workspace (the
    library's fixed device scratch array is used instead).  Returns
    (loss[1], grad[n]) float64 tensors."""
    pair, keep = make_pair(R, I, m, mask, var, flat, bg_degree)
    if not R.is_cuda:
        raise ValueError("loss_grad_noalloc takes device tensors")
    theta = theta.to(device=R.device, dtype=torch.float64).contiguous()
    n = n_params(m, bg_degree)
    if theta.numel() != n:
        raise ValueError(f"theta must have {n} entries")
    loss = torch.empty(1, dtype=torch.float64, device=R.device)
    grad = torch.empty(n, dtype=torch.float64, device=R.device)
    st = lib.dia_loss_grad_noalloc(ctypes.byref(pair), ctypes.byref(spec), _ptr(theta),
                                   _ptr(loss), _ptr(grad), _stream(stream))
    _check(st, "dia_loss_grad_noalloc")
    return loss, grad


def diff_image(R, I, m, theta, ws=None, stream=None, bg_degree=0, kernel_degree=0):
    pair, keep = make_pair(R, I, m, bg_degree=bg_degree, kernel_degree=kernel_degree)
    theta = theta.to(device=R.device, dtype=torch.float64).contiguous()
    ws = ws if ws is not None else pair_workspace(pair, device=R.device)
    h = m // 2
    out = torch.empty((pair.H - 2 * h, pair.W - 2 * h), dtype=torch.float32, device=R.device)
    _check(lib.dia_diff_image(ctypes.byref(pair), _ptr(theta), _ptr(out), _ptr(ws), ws.numel(),
                              _stream(stream)), "dia_diff_image")
    return out


def diff_image_tc(R, I, m, theta, ws=None, stream=None):
    """dia_diff_image_tc: the difference image with the correlation on the
    tensor cores (split bf16, float32 accumulation; constant background)."""
    pair, keep = make_pair(R, I, m)
    theta = theta.to(device=R.device, dtype=torch.float64).contiguous()
    ws = ws if ws is not None else workspace(pair.H, pair.W, m, pair.ld, device=R.device)
    h = m // 2
    out = torch.empty((pair.H - 2 * h, pair.W - 2 * h), dtype=torch.float32, device=R.device)
    _check(lib.dia_diff_image_tc(ctypes.byref(pair), _ptr(theta), _ptr(out), _ptr(ws),
                                 ws.numel(), _stream(stream)), "dia_diff_image_tc")
    return out


def loss_grad_tc(R, I, m, theta, spec: LossSpec, mask=None, var=None, flat=None, stream=None):
    """dia_loss_grad_tc: the evaluation with both contractions on the tensor
    cores.  Returns (loss[1], grad[n]) float64 device tensors."""
    pair, keep = make_pair(R, I, m, mask, var, flat)
    if not R.is_cuda:
        raise ValueError("loss_grad_tc takes device tensors")
    theta = theta.to(device=R.device, dtype=torch.float64).contiguous()
    nb = lib.dia_tc_workspace_size(pair.H, pair.W, pair.ld, m)
    if nb == 0:
        raise DiaError(DIA_ERR_ARG, "dia_tc_workspace_size")
    ws = torch.empty(nb, dtype=torch.uint8, device=R.device)
    loss = torch.empty(1, dtype=torch.float64, device=R.device)
    grad = torch.empty(m * m + 1, dtype=torch.float64, device=R.device)
    st = lib.dia_loss_grad_tc(ctypes.byref(pair), ctypes.byref(spec), _ptr(theta), _ptr(loss),
                              _ptr(grad), _ptr(ws), nb, _stream(stream))
    _check(st, "dia_loss_grad_tc")
    return loss, grad


def fit(R, I, m, spec: LossSpec, opts: Opts = None, mask=None, var=None, flat=None,
        theta0=None, want_diff=True, want_mask=False, ws=None, stream=None, check=True,
        bg_degree=0, kernel_degree=0):
    """dia_fit.  Tensors on one CUDA device, or all on the host (the library
    then stages them through the workspace and returns host tensors).
    ``bg_degree``: degree of the polynomial background (Eq. 18);
    ``kernel_degree``: degree of a spatially varying kernel (0: one kernel).
    Returns dict(theta, K, b0, diff, mask, info)."""
    pair, keep = make_pair(R, I, m, mask, var, flat, bg_degree, kernel_degree)
    host = pair.mem == MEM_HOST
    dev = R.device
    opts = opts if opts is not None else default_opts()
    o = Opts.from_buffer_copy(opts)
    th0 = None
    if theta0 is not None:
        th0 = np.ascontiguousarray(np.asarray(theta0, dtype=np.float64))
        o.theta0 = th0.ctypes.data
        o.init = 2
    clip = o.clip_passes > 0 or want_mask
    if ws is None:
        ws = pair_workspace(pair, clip, device=None if host else dev)
    n = n_params(m, bg_degree, kernel_degree)
    if th0 is not None and th0.size != n:
        raise ValueError(f"theta0 must have {n} entries")
    h = m // 2
    kw = dict(device=dev)
    if host:
        kw["pin_memory"] = R.is_pinned()
    theta = torch.empty(n, dtype=torch.float64, **kw)
    K = torch.empty((m, m), dtype=torch.float32, **kw)
    b0 = torch.empty(1, dtype=torch.float32, **kw)
    diff = torch.empty((pair.H - 2 * h, pair.W - 2 * h), dtype=torch.float32, **kw) \
        if want_diff else None
    mk = torch.empty((pair.H, pair.ld), dtype=torch.uint8, **kw)[:, :pair.W] \
        if want_mask else None
    info = FitInfo()
    st = lib.dia_fit(ctypes.byref(pair), ctypes.byref(spec), ctypes.byref(o), _ptr(theta),
                     _ptr(K), _ptr(b0), _ptr(diff), _ptr(mk), ctypes.byref(info), _ptr(ws),
                     ws.numel(), _stream(stream))
    if check and st not in (DIA_OK, DIA_ERR_MAXITER):
        raise DiaError(st, "dia_fit")
    return dict(theta=theta, K=K, b0=b0, diff=diff, mask=mk, info=info.as_dict(), status=st)


def fit_batch(items, spec: LossSpec, opts: Opts = None, want_diff=False, ws=None, stream=None):
    """dia_fit_batch over a list of dicts {R, I, m, mask?, var?, flat?,
    bg_degree?} of device tensors.  Returns dict(thetas=[float64 tensors],
    diffs=[...] or None, infos=[dict], status)."""
    n = len(items)
    pairs = (Pair * n)()
    keep = []
    for i, it in enumerate(items):
        p, k = make_pair(it["R"], it["I"], it["m"], it.get("mask"), it.get("var"), it.get("flat"),
                         it.get("bg_degree", 0))
        if p.mem != MEM_DEVICE:
            raise ValueError("fit_batch takes device tensors")
        pairs[i] = p
        keep.append(k)
    opts = opts if opts is not None else default_opts()
    dev = items[0]["R"].device
    need = lib.dia_batch_workspace_size(pairs, n, ctypes.byref(opts))
    if need == 0:
        raise DiaError(DIA_ERR_ARG, "dia_batch_workspace_size")
    if ws is None or ws.numel() < need:
        ws = torch.empty(need, dtype=torch.uint8, device=dev)
    sizes = [n_params(it["m"], it.get("bg_degree", 0)) for it in items]
    theta = torch.empty(sum(sizes), dtype=torch.float64, device=dev)
    diffs = None
    dptr = None
    if want_diff:
        diffs = [torch.empty((it["R"].shape[0] - 2 * (it["m"] // 2),
                              it["R"].shape[1] - 2 * (it["m"] // 2)), dtype=torch.float32,
                             device=dev) for it in items]
        dptr = (ctypes.c_void_p * n)(*[d.data_ptr() for d in diffs])
    infos = (FitInfo * n)()
    st = lib.dia_fit_batch(pairs, n, ctypes.byref(spec), ctypes.byref(opts), _ptr(theta),
                           dptr, infos, _ptr(ws), ws.numel(), _stream(stream))
    if st not in (DIA_OK, DIA_ERR_MAXITER):
        raise DiaError(st, "dia_fit_batch")
    thetas = list(torch.split(theta, sizes))
    return dict(thetas=thetas, diffs=diffs, infos=[f.as_dict() for f in infos], status=st,
                ws=ws)


class DiaLossGrad(torch.autograd.Function):
    """L(theta) with the hand-written fused backward (Sec. 2.3).

    forward runs one fused pass that returns the loss and keeps only the
    gradient vector (len(theta) float64 values): no model image or other
    activation is stored; backward scales that gradient by grad_output."""

    @staticmethod
    def forward(ctx, theta, R, I, m, spec, mask=None, var=None, flat=None, bg_degree=0):
        loss, grad = loss_grad(R, I, m, theta.detach(), spec, mask, var, flat,
                               bg_degree=bg_degree)
        ctx.save_for_backward(grad)
        return loss.reshape(()).to(theta.dtype)

    @staticmethod
    def backward(ctx, gout):
        (grad,) = ctx.saved_tensors
        return (gout * grad).to(gout.dtype), None, None, None, None, None, None, None, None


def dia_loss(theta, R, I, m, spec, mask=None, var=None, flat=None, bg_degree=0):
    return DiaLossGrad.apply(theta, R, I, m, spec, mask, var, flat, bg_degree)

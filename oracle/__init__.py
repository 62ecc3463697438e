"""FP64 CPU oracle for the DIA kernel fit of PyTorchDIA (arXiv 2104.13715).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this package.  The product library never
loads it and shares no code with it: the direct loops live in ``dia_oracle.c``
(compiled here with the system C compiler), the linear algebra is numpy.

Pieces (each cites the passage it follows):

* :func:`model`, :func:`loss_grad`, :func:`pixel_terms` -- the image model
  (Sec. 2.1, Eq. 2), the noise models (Eq. 6, Eq. 7) and the loss (Eq. 8,
  Eq. 13 with the Huber rho of Eq. 12 or a Cauchy rho as the Student-t drop-in
  named in Sec. 2.4), by direct loops in FP64.
* :func:`gram`, :func:`normal_solve` -- the Bramich (2008) normal equations
  for the fixed-variance chi^2 (Sec. 1 and Sec. 2.1): A = sum w phi phi^T,
  b = sum w phi I with phi_p = [R window of p, background basis at p], solved
  by Cholesky.
* :func:`background_basis` -- the polynomial background of Sec. 2.6 (Eq. 18)
  in the normalised coordinates of Eq. 19; degree 0 is the constant B0.  Every
  function taking theta reads the degree from its length, m*m + (d+1)(d+2)/2.
* :func:`laplacian`, :func:`penalty` -- the kernel regulariser of Sec. 2.7
  (Eq. 20, Eq. 21): lam * N_data * theta^T L^T L theta with L the Laplacian of
  the kernel-pixel graph (4-connectivity); loss_grad, normal_solve, hessian
  and newton take it through ``reg_lambda``.
* :func:`svk_model`, :func:`svk_loss_grad`, :func:`svk_normal_solve`,
  :func:`svk_hessian`, :func:`svk_newton` -- a
  spatially varying kernel (each kernel pixel a polynomial of degree dk in the
  coordinates of Eq. 19, the Bramich et al. 2013 form the paper cites in
  Sec. 1), in numpy for small images.
* :func:`newton` -- for the losses that are not quadratic in theta: Newton
  steps with the exact Hessian sum_p l''(M_p) phi_p phi_p^T (M is linear in
  theta), Levenberg damping where it is not positive definite, backtracking
  on the FP64 loss.
* :func:`diff_image`, :func:`sigma_clip`, :func:`fit_clipped` -- the
  difference image I - M and the kappa-sigma clipping of B08 (Sec. 2.4,
  Sec. 4.2).

Conventions: theta = [K row-major over (row offset, column offset), b] with b
= [B0] or the coefficients b_00, b_01, ..., b_0d, b_10, ..., b_d0 of Eq. 18 (the
power of xi running fastest); eta = (x - x_c)/N_x, xi = (y - y_c)/N_y with x
the column and y the row of the full image, x_c = (W - 1)/2, y_c = (H - 1)/2,
N_x = W, N_y = H;
``K[a, b]`` multiplies ``R[i - h + a, j - h + b]`` for the target pixel
(i, j), with h = m // 2, so ``a = b = h`` is the kernel centre and a +1 pixel
shift of the target in x and y gives a delta at ``a = b = h - 1`` (Sec. 3.4
test iii).  Only the valid region i, j in [h, N - h) enters the fit.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dia_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_dia_oracle.so")
_lock = threading.Lock()
_lib = None

RHO = {"gauss": 0, "huber": 1, "cauchy": 2}
NOISE = {"fixed": 0, "ccd": 1, "emccd": 2}


def build(force: bool = False) -> str:
    """Compile ``dia_oracle.c`` into ``_dia_oracle.so`` (plain gcc, OpenMP)."""
    if not force and os.path.exists(_LIB_PATH) and \
            os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        up = ctypes.POINTER(ctypes.c_uint8)
        i = ctypes.c_int
        lib.oracle_model.argtypes = [dp, i, i, i, i, i, dp, dp, i]
        lib.oracle_model.restype = i
        lib.oracle_pixel_terms.argtypes = [dp, up, dp, dp, i, i, i, i, dp, dp,
                                           dp, dp, dp, dp]
        lib.oracle_pixel_terms.restype = i
        lib.oracle_loss_grad.argtypes = [dp, dp, up, dp, dp, i, i, i, i, i, dp, dp,
                                         dp, dp, i]
        lib.oracle_loss_grad.restype = i
        lib.oracle_ndata.argtypes = [up, i, i, i, i]
        lib.oracle_ndata.restype = ctypes.c_longlong
        lib.oracle_design_rows.argtypes = [dp, i, i, i, i, i, i, i, dp, i, dp, dp, i]
        lib.oracle_design_rows.restype = i
        _lib = lib
        return lib


@dataclass
class LossSpec:
    """Loss choice: rho in {gauss, huber, cauchy}, variance model in
    {fixed, ccd, emccd} (Eq. 6, Eq. 7), and their constants."""
    rho: str = "gauss"
    noise: str = "fixed"
    sigma0: float = 0.0        # read noise (image units), CCD model
    gain: float = 1.0          # G (CCD) or G_total (EMCCD)
    excess: float = 2.0        # EMCCD excess noise factor E (Sec. 2.1)
    huber_c: float = 1.345     # Huber threshold (Sec. 2.4)
    var: float = 1.0           # scalar fixed variance when no map is given
    var_floor: float = 1e-6    # lower clamp of a model-dependent variance

    def params(self) -> np.ndarray:
        return np.array([RHO[self.rho], NOISE[self.noise], self.sigma0, self.gain,
                         self.excess, self.huber_c, self.var, self.var_floor],
                        dtype=np.float64)


def _d(a):
    if a is None:
        return None
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a, ctype=ctypes.c_double):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _u8(a):
    if a is None:
        return None
    return np.ascontiguousarray(a, dtype=np.uint8)


def _shape(R, m):
    H, W = R.shape
    if m < 1 or m % 2 == 0 or m > min(H, W):
        raise ValueError(f"kernel side m={m} must be odd and <= image side")
    return H, W


def n_background(deg: int) -> int:
    """Coefficients of the degree-d polynomial of Eq. 18: (d+1)(d+2)/2."""
    return (deg + 1) * (deg + 2) // 2


def n_params(m: int, deg: int = 0) -> int:
    return m * m + n_background(deg)


def degree_of(theta, m) -> int:
    """Background degree implied by len(theta) = m*m + (d+1)(d+2)/2."""
    nb = len(theta) - m * m
    for d in range(10):
        if n_background(d) == nb:
            return d
    raise ValueError(f"theta of length {len(theta)} fits no background degree for m={m}")


def background_basis(shape, m, deg):
    """The basis eta^p xi^q of Eq. 18 over the valid region, shape (Hv, Wv,
    (d+1)(d+2)/2), in the coefficient order of theta; eta, xi of Eq. 19 on the
    full image's pixel grid (column x, row y), centred at ((W-1)/2, (H-1)/2)
    and scaled by W and H."""
    H, W = shape
    h = m // 2
    y = np.arange(h, H - h, dtype=np.float64)
    x = np.arange(h, W - h, dtype=np.float64)
    xi = (y - 0.5 * (H - 1)) / H
    eta = (x - 0.5 * (W - 1)) / W
    cols = []
    for p in range(deg + 1):
        for q in range(deg - p + 1):
            cols.append(np.outer(xi ** q, eta ** p))
    return np.stack(cols, axis=-1)


def laplacian(m: int, deg: int = 0) -> np.ndarray:
    """Laplacian matrix of the kernel-pixel graph (Sec. 2.7, Eq. 21), of size
    n_params(m, deg) square: L[u, u] = number of kernel pixels adjacent to u,
    L[u, v] = -1 for adjacent u, v (sharing an edge: 4-connectivity), zero in
    the rows and columns of the background coefficients."""
    n = n_params(m, deg)
    L = np.zeros((n, n))
    for a in range(m):
        for b in range(m):
            u = a * m + b
            for da, db in ((-1, 0), (1, 0), (0, -1), (0, 1)):
                aa, bb = a + da, b + db
                if 0 <= aa < m and 0 <= bb < m:
                    L[u, aa * m + bb] = -1.0
                    L[u, u] += 1.0
    return L


def penalty(theta, m, lam, n_data):
    """The regulariser of Eq. 20, lam * N_data * theta^T L^T L theta, with its
    gradient and Hessian (L of Eq. 21)."""
    th = np.asarray(theta, dtype=np.float64)
    L = laplacian(m, degree_of(th, m))
    LtL = L.T @ L
    c = lam * n_data
    return c * th @ LtL @ th, 2.0 * c * LtL @ th, 2.0 * c * LtL


def ndata(shape, m, mask=None) -> int:
    """Valid, unmasked pixel count N_data = (N - 2h)^2 without a mask (Sec. 2.1)."""
    H, W = shape
    mk = _u8(mask)
    return int(_load().oracle_ndata(_ptr(mk, ctypes.c_uint8), H, W, W, m))


def model(R, theta, m, nthreads: int = 0) -> np.ndarray:
    """Model image M = R (x) K + B over the valid region (Eq. 2; B the constant
    B0 or the polynomial of Eq. 18, by the length of theta)."""
    R = _d(R)
    H, W = _shape(R, m)
    th = _d(theta)
    h = m // 2
    out = np.empty((H - 2 * h, W - 2 * h), dtype=np.float64)
    rc = _load().oracle_model(_ptr(R), H, W, W, m, degree_of(th, m), _ptr(th), _ptr(out),
                              nthreads)
    if rc:
        raise ValueError("oracle_model: bad arguments")
    return out


def pixel_terms(I, M, m, spec: LossSpec, mask=None, var=None, flat=None):
    """Per-pixel (loss, dl/dM, d2l/dM2, z) over the valid region; masked pixels
    get zero loss and derivatives (z is still reported)."""
    I = _d(I)
    H, W = I.shape
    h = m // 2
    M = _d(M)
    assert M.shape == (H - 2 * h, W - 2 * h)
    outs = [np.empty_like(M) for _ in range(4)]
    rc = _load().oracle_pixel_terms(_ptr(I), _ptr(_u8(mask), ctypes.c_uint8),
                                    _ptr(_d(var)), _ptr(_d(flat)), H, W, W, m,
                                    _ptr(spec.params()), _ptr(M),
                                    *[_ptr(o) for o in outs])
    if rc:
        raise ValueError("oracle_pixel_terms: bad arguments")
    return tuple(outs)


def loss_grad(R, I, m, theta, spec: LossSpec = None, mask=None, var=None, flat=None,
              nthreads: int = 0, reg_lambda: float = 0.0):
    """FP64 loss L(theta) and gradient dL/dtheta (Eq. 8 / Eq. 13, summed over the
    unmasked valid pixels; with reg_lambda > 0, plus the regulariser of Eq. 20).
    Returns (L, grad[len(theta)])."""
    spec = spec or LossSpec()
    R = _d(R)
    I = _d(I)
    H, W = _shape(R, m)
    assert I.shape == R.shape
    th = _d(theta)
    deg = degree_of(th, m)
    loss = np.zeros(1)
    grad = np.zeros(n_params(m, deg))
    mk = _u8(mask)
    vv = _d(var)
    ff = _d(flat)
    rc = _load().oracle_loss_grad(_ptr(R), _ptr(I), _ptr(mk, ctypes.c_uint8), _ptr(vv),
                                  _ptr(ff), H, W, W, m, deg, _ptr(spec.params()), _ptr(th),
                                  _ptr(loss), _ptr(grad), nthreads)
    if rc:
        raise ValueError(f"oracle_loss_grad failed ({rc})")
    if reg_lambda:
        pv, pg, _ = penalty(th, m, reg_lambda, ndata(R.shape, m, mask))
        return float(loss[0]) + pv, grad + pg
    return float(loss[0]), grad


def loss(R, I, m, theta, spec: LossSpec = None, mask=None, var=None, flat=None):
    return loss_grad(R, I, m, theta, spec, mask, var, flat)[0]


def _windows(R, m):
    return np.lib.stride_tricks.sliding_window_view(R, (m, m))


def gram(R, m, weights, rhs=None, block_rows: int = 0, deg: int = 0):
    """A = sum_p w_p phi_p phi_p^T and (optionally) b = sum_p rhs_p phi_p, where
    phi_p = [R window of valid pixel p (m*m, row-major), background basis at p
    (Eq. 18; [1] for degree 0)].  ``weights`` and ``rhs`` are arrays over the
    valid region.  This is the B08 normal matrix when w = 1/sigma^2 and
    rhs = I/sigma^2 (Sec. 1).  The rows phi_p and w_p phi_p of a block of image
    rows are laid out by ``oracle_design_rows`` (C, threaded copy) and the
    block's sum is one matrix product; blocks (about 2^25 doubles each unless
    ``block_rows`` is given) are added in row order."""
    R = _d(R)
    H, W = _shape(R, m)
    h = m // 2
    Hv, Wv = H - 2 * h, W - 2 * h
    n = n_params(m, deg)
    w_all = np.ascontiguousarray(weights, dtype=np.float64)
    assert w_all.shape == (Hv, Wv)
    if block_rows <= 0:
        block_rows = max(1, (1 << 25) // (Wv * n))
    lib = _load()
    A = np.zeros((n, n))
    b = np.zeros(n) if rhs is not None else None
    phi = np.empty((min(block_rows, Hv) * Wv, n))
    phiw = np.empty_like(phi)
    for y0 in range(0, Hv, block_rows):
        y1 = min(Hv, y0 + block_rows)
        k = (y1 - y0) * Wv
        rc = lib.oracle_design_rows(_ptr(R), H, W, W, m, deg, y0, y1, _ptr(w_all), Wv,
                                    _ptr(phi), _ptr(phiw), 0)
        if rc:
            raise ValueError("oracle_design_rows: bad arguments")
        A += phiw[:k].T @ phi[:k]
        if rhs is not None:
            b += phi[:k].T @ np.asarray(rhs[y0:y1], dtype=np.float64).reshape(-1)
    return (A, b) if rhs is not None else A


class Degenerate(RuntimeError):
    """The normal matrix / Hessian is singular (e.g. constant R, all masked)."""


def _valid(a, m):
    h = m // 2
    return a[h:a.shape[0] - h, h:a.shape[1] - h]


def normal_solve(R, I, m, mask=None, var=None, var_scalar: float = 1.0,
                 reg_lambda: float = 0.0, deg: int = 0):
    """B08 linear least squares for the fixed-variance chi^2: solve A theta = b
    by Cholesky (Sec. 1; Sec. 2.1 'fixed estimates for sigma').  With
    reg_lambda > 0 the minimum of chi^2/2 + the regulariser of Eq. 20:
    (A + 2 lam N_data L^T L) theta = b."""
    R = _d(R)
    I = _d(I)
    H, W = _shape(R, m)
    Iv = _valid(I, m)
    w = np.ones_like(Iv) / var_scalar if var is None else 1.0 / _valid(_d(var), m)
    if mask is not None:
        w = w * (_valid(np.asarray(mask), m) != 0)
    A, b = gram(R, m, w, w * Iv, deg=deg)
    if reg_lambda:
        A = A + penalty(np.zeros(n_params(m, deg)), m, reg_lambda, ndata(R.shape, m, mask))[2]
    try:
        L = np.linalg.cholesky(A)
    except np.linalg.LinAlgError as e:
        raise Degenerate(str(e))
    y = np.linalg.solve(L, b)
    return np.linalg.solve(L.T, y)


def hessian(R, I, m, theta, spec: LossSpec, mask=None, var=None, flat=None,
            reg_lambda: float = 0.0):
    """Exact Hessian sum_p l''(M_p) phi_p phi_p^T (M is linear in theta), plus
    that of the regulariser of Eq. 20 when reg_lambda > 0."""
    M = model(R, theta, m)
    _, _, d2, _ = pixel_terms(I, M, m, spec, mask, var, flat)
    Hm = gram(R, m, d2, deg=degree_of(theta, m))
    if reg_lambda:
        Hm = Hm + penalty(theta, m, reg_lambda, ndata(np.shape(R), m, mask))[2]
    return Hm


def newton(R, I, m, theta0, spec: LossSpec, mask=None, var=None, flat=None,
           max_iter: int = 50, rtol: float = 1e-13, verbose: bool = False,
           reg_lambda: float = 0.0):
    """Damped Newton iteration on the FP64 loss to its stationary point.

    Step: solve (H + lam diag(H)) d = -g with lam = 0 unless H is not positive
    definite; backtrack on the loss (Armijo, c = 1e-4).  Stops when the step is
    below rtol relative to theta or the loss no longer decreases."""
    th = _d(theta0).copy()
    L, g = loss_grad(R, I, m, th, spec, mask, var, flat, reg_lambda=reg_lambda)
    for it in range(max_iter):
        Hm = hessian(R, I, m, th, spec, mask, var, flat, reg_lambda=reg_lambda)
        dH = np.diag(Hm).copy()
        if np.all(dH == 0):
            raise Degenerate("zero Hessian")
        lam = 0.0
        while True:
            try:
                C = np.linalg.cholesky(Hm + lam * np.diag(np.abs(dH) + 1e-300))
                break
            except np.linalg.LinAlgError:
                lam = 1e-6 if lam == 0.0 else lam * 10.0
                if lam > 1e12:
                    raise Degenerate("Hessian not positive definite")
        d = -np.linalg.solve(C.T, np.linalg.solve(C, g))
        t = 1.0
        slope = float(g @ d)
        while True:
            Lt, gt = loss_grad(R, I, m, th + t * d, spec, mask, var, flat, reg_lambda=reg_lambda)
            if Lt <= L + 1e-4 * t * slope or t < 1e-12:
                break
            t *= 0.5
        step = t * d
        th = th + step
        dec = L - Lt
        L, g = Lt, gt
        if verbose:
            print(f"newton it={it} L={L:.17g} |step|={np.max(np.abs(step)):.3e}")
        if np.max(np.abs(step)) <= rtol * (1.0 + np.max(np.abs(th))) or dec <= 0.0:
            break
    return th


def fit(R, I, m, spec: LossSpec = None, mask=None, var=None, flat=None,
        theta0=None, max_iter: int = 50, deg: int = 0):
    """The minimiser of the loss.  Fixed-variance Gaussian: the B08 normal
    solve.  Otherwise: Newton from theta0 (default: the normal solve with the
    scalar variance, which is the B08 first iteration).  ``deg``: background
    degree (Eq. 18) when theta0 is not given."""
    spec = spec or LossSpec()
    if theta0 is not None:
        deg = degree_of(theta0, m)
    if spec.rho == "gauss" and spec.noise == "fixed":
        return normal_solve(R, I, m, mask, var, spec.var, deg=deg)
    if theta0 is None:
        theta0 = normal_solve(R, I, m, mask, var if spec.noise == "fixed" else None,
                              spec.var if spec.noise == "fixed" else 1.0, deg=deg)
    return newton(R, I, m, theta0, spec, mask, var, flat, max_iter=max_iter)


def diff_image(R, I, m, theta) -> np.ndarray:
    """Difference image D = I - M over the valid region (Sec. 1)."""
    return _valid(_d(I), m) - model(R, theta, m)


def sigma_clip(R, I, m, theta, spec: LossSpec, mask=None, var=None, flat=None,
               kappa: float = 5.0) -> np.ndarray:
    """Mask (full image, uint8, 1 = use) after clipping |z| > kappa on the
    valid region, z = (I - M)/sigma (B08 clipping, Sec. 4.2).  Clipping is
    cumulative: a pixel already masked stays masked."""
    I = _d(I)
    H, W = I.shape
    h = m // 2
    M = model(R, theta, m)
    _, _, _, z = pixel_terms(I, M, m, spec, None, var, flat)
    out = np.ones((H, W), np.uint8) if mask is None else np.array(mask, np.uint8)
    v = out[h:H - h, h:W - h]
    v[np.abs(z) > kappa] = 0
    return out


def fit_clipped(R, I, m, spec: LossSpec, mask=None, var=None, flat=None,
                passes: int = 3, kappa: float = 5.0, theta0=None, deg: int = 0):
    """Fit, then `passes` times: clip at kappa and refit from the current theta.
    Returns (theta, mask)."""
    th = fit(R, I, m, spec, mask, var, flat, theta0, deg=deg)
    mk = None if mask is None else np.array(mask, np.uint8)
    for _ in range(passes):
        mk = sigma_clip(R, I, m, th, spec, mk, var, flat, kappa)
        th = fit(R, I, m, spec, mk, var, flat, theta0=th)
    return th, mk


# ---------------------------------------------------------------------------
# Spatially varying kernel.  The paper mentions this extension of DIA (Sec. 1,
# citing Alard 2000 and Bramich et al. 2013) without implementing it; the
# reading taken here is the Bramich et al. form: every kernel pixel varies over
# the image as a polynomial of degree dk in the normalised coordinates of
# Eq. 19,
#     K_ab(x, y) = sum_{p+q <= dk} K_pq[a][b] eta^p xi^q,
# evaluated at the output pixel, so that
#     M = sum_pq eta^p xi^q (R (x) K_pq) + B(x, y)
# stays linear in theta = [K_00, K_01, ..., K_dk0 (m*m each, the coefficient
# order of Eq. 18), background coefficients].  dk = 0 is the constant kernel.
# Plain numpy over the valid region (small images only).
# ---------------------------------------------------------------------------
def svk_split(theta, m, dk):
    """(list of the n_background(dk) kernel coefficient arrays m x m, background
    coefficients) of a spatially varying kernel theta."""
    th = np.asarray(theta, dtype=np.float64)
    nk = n_background(dk)
    ks = [th[c * m * m:(c + 1) * m * m].reshape(m, m) for c in range(nk)]
    bg = th[nk * m * m:]
    degree_of(np.concatenate([np.zeros(m * m), bg]), m)   # validates the background length
    return ks, bg


def svk_model(R, theta, m, dk) -> np.ndarray:
    """Model image with the spatially varying kernel over the valid region."""
    R = _d(R)
    H, W = _shape(R, m)
    ks, bg = svk_split(theta, m, dk)
    win = _windows(R, m)                          # (Hv, Wv, m, m): R[y + a][x + b]
    phi = background_basis((H, W), m, dk)         # (Hv, Wv, nk): eta^p xi^q
    M = np.zeros(win.shape[:2])
    for c, K in enumerate(ks):
        M += phi[..., c] * np.einsum("yxab,ab->yx", win, K)
    B = background_basis((H, W), m, degree_of(np.concatenate([np.zeros(m * m), bg]), m))
    return M + B @ bg


def svk_loss_grad(R, I, m, theta, dk, spec: LossSpec = None, mask=None, var=None, flat=None):
    """FP64 loss and gradient for the spatially varying kernel: the per-pixel
    terms of Eq. 8 / Eq. 13 at M = svk_model, dL/dK_pq[a][b] = sum_p g_p eta^p
    xi^q R[y + a][x + b], dL/db = sum_p g_p (background basis)."""
    spec = spec or LossSpec()
    R = _d(R)
    H, W = _shape(R, m)
    M = svk_model(R, theta, m, dk)
    ell, g, _, _ = pixel_terms(I, M, m, spec, mask, var, flat)
    win = _windows(R, m)
    phi = background_basis((H, W), m, dk)
    ks, bg = svk_split(theta, m, dk)
    grads = [np.einsum("yx,yxab->ab", g * phi[..., c], win).ravel() for c in range(len(ks))]
    B = background_basis((H, W), m, degree_of(np.concatenate([np.zeros(m * m), bg]), m))
    grads.append(np.einsum("yx,yxk->k", g, B))
    return float(np.sum(ell)), np.concatenate(grads)


def svk_normal_solve(R, I, m, dk, deg: int = 0, mask=None, var=None, var_scalar: float = 1.0):
    """The fixed-variance chi^2 minimum for the spatially varying kernel: the
    design row of pixel p is [eta^p xi^q R window of p for each (p, q), background
    basis at p]; A = sum w phi phi^T, b = sum w phi I, solved by Cholesky."""
    R = _d(R)
    I = _d(I)
    H, W = _shape(R, m)
    Iv = _valid(I, m)
    w = np.ones_like(Iv) / var_scalar if var is None else 1.0 / _valid(_d(var), m)
    if mask is not None:
        w = w * (_valid(np.asarray(mask), m) != 0)
    win = _windows(R, m).reshape(Iv.shape[0], Iv.shape[1], m * m)
    phi = background_basis((H, W), m, dk)
    B = background_basis((H, W), m, deg)
    cols = [phi[..., c:c + 1] * win for c in range(phi.shape[-1])] + [B]
    X = np.concatenate(cols, axis=-1).reshape(-1, phi.shape[-1] * m * m + B.shape[-1])
    wv = w.reshape(-1)
    A = (X * wv[:, None]).T @ X
    b = X.T @ (wv * Iv.reshape(-1))
    try:
        L = np.linalg.cholesky(A)
    except np.linalg.LinAlgError as e:
        raise Degenerate(str(e))
    return np.linalg.solve(L.T, np.linalg.solve(L, b))


def svk_hessian(R, I, m, theta, dk, spec: LossSpec, mask=None, var=None, flat=None):
    """Exact Hessian of the spatially varying kernel's loss: sum_p l''(M_p)
    phi_p phi_p^T with phi_p the design row of svk_normal_solve (M is linear in
    theta)."""
    R = _d(R)
    H, W = _shape(R, m)
    M = svk_model(R, theta, m, dk)
    _, _, d2, _ = pixel_terms(I, M, m, spec, mask, var, flat)
    ks, bg = svk_split(theta, m, dk)
    deg = degree_of(np.concatenate([np.zeros(m * m), bg]), m)
    win = _windows(R, m).reshape(M.shape[0], M.shape[1], m * m)
    phi = background_basis((H, W), m, dk)
    B = background_basis((H, W), m, deg)
    cols = [phi[..., c:c + 1] * win for c in range(phi.shape[-1])] + [B]
    X = np.concatenate(cols, axis=-1).reshape(-1, phi.shape[-1] * m * m + B.shape[-1])
    return (X * d2.reshape(-1)[:, None]).T @ X


def svk_newton(R, I, m, theta0, dk, spec: LossSpec, mask=None, var=None, flat=None,
               max_iter: int = 50, rtol: float = 1e-13):
    """Damped Newton on the spatially varying kernel's FP64 loss (the steps of
    :func:`newton`: Levenberg damping where the Hessian is not positive
    definite, Armijo backtracking)."""
    th = _d(theta0).copy()
    L, g = svk_loss_grad(R, I, m, th, dk, spec, mask, var, flat)
    for _ in range(max_iter):
        Hm = svk_hessian(R, I, m, th, dk, spec, mask, var, flat)
        dH = np.diag(Hm).copy()
        if np.all(dH == 0):
            raise Degenerate("zero Hessian")
        lam = 0.0
        while True:
            try:
                Lc = np.linalg.cholesky(Hm + lam * np.diag(np.abs(dH) + 1e-300))
                break
            except np.linalg.LinAlgError:
                lam = 1e-6 if lam == 0.0 else lam * 10.0
                if lam > 1e12:
                    raise Degenerate("Hessian not positive definite")
        d = -np.linalg.solve(Lc.T, np.linalg.solve(Lc, g))
        t, slope = 1.0, float(g @ d)
        while True:
            Lt, gt = svk_loss_grad(R, I, m, th + t * d, dk, spec, mask, var, flat)
            if Lt <= L + 1e-4 * t * slope or t < 1e-12:
                break
            t *= 0.5
        step = t * d
        th = th + step
        dec = L - Lt
        L, g = Lt, gt
        if np.max(np.abs(step)) <= rtol * (1.0 + np.max(np.abs(th))) or dec <= 0.0:
            break
    return th

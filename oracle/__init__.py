"""FP64 CPU oracle for the Domain Transform Solver -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never does, and this package imports nothing from it.

The arithmetic lives in ``dts_oracle.c`` (plain double-precision loops, each
function citing the passage of the paper it follows); this module only
marshals numpy arrays.  Array conventions: images are ``(H, W)`` float64,
guides ``(C, H, W)`` float64, C-contiguous.
"""
import ctypes
import os

import numpy as np

from . import build as _build

NORM_L1, NORM_L2 = 0, 1
UPDATE_GD, UPDATE_JACOBI = 0, 1
CONF_PLAIN, CONF_SUPPORT = 0, 1
KERNEL_RF, KERNEL_BOX = 0, 1

_lib = None
_dp = ctypes.POINTER(ctypes.c_double)


def _load():
    global _lib
    if _lib is None:
        # DTS_ORACLE_SO: a separately compiled copy of this oracle (the mutation test builds copies
        # with planted mistakes and runs the pins against them)
        path = os.environ.get("DTS_ORACLE_SO") or _build.build()
        lib = ctypes.CDLL(path)
        i, d, p = ctypes.c_int, ctypes.c_double, _dp
        lib.orc_schedule.argtypes = [d, i, p, p]
        lib.orc_distances.argtypes = [i, i, i, p, d, d, i, p, p]
        lib.orc_causal.argtypes = [i, p, ctypes.c_long, p, ctypes.c_long, d]
        lib.orc_anticausal.argtypes = [i, p, ctypes.c_long, p, ctypes.c_long, d]
        lib.orc_row_pass.argtypes = [i, i, p, p, d]
        lib.orc_col_pass.argtypes = [i, i, p, p, d]
        lib.orc_filter.argtypes = [i, i, p, p, i, p, p, p]
        lib.orc_support.argtypes = [i, i, p, p, d, p, p]
        lib.orc_confidence.argtypes = [i, i, p, p, i, p, p, d, p]
        lib.orc_box_filter.argtypes = [i, i, p, p, i, p, p, p]
        lib.orc_solve_kernel.argtypes = [i, i, p, p, p, p, p, d, d, d, i, i, i, d, i, i, p, p]
        lib.orc_solve_cg.argtypes = [i, i, p, p, p, p, p, d, d, i, i, p]
        lib.orc_solve.argtypes = [i, i, p, p, p, p, p, d, d, d, i, i, i, i, p, p]
        lib.orc_solve.restype = i
        lib.orc_filter_adjoint.argtypes = [i, i, p, p, i, p, p, p, p, p, p]
        lib.orc_distances_adjoint.argtypes = [i, i, i, p, d, d, i, p, p, p, p, p]
        lib.orc_solve_backward.argtypes = [i, i, i, p, d, d, i, p, p, p, d, d, i, i, i, d, i, p, p, p, p, p]
        lib.orc_solve_backward.restype = i
        lib.orc_num_threads.restype = i
        lib.orc_set_num_threads.argtypes = [i]
        _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(_dp)


def num_threads() -> int:
    """OpenMP threads the oracle uses."""
    return _load().orc_num_threads()


def set_num_threads(n: int) -> None:
    _load().orc_set_num_threads(int(n))


def schedule(sigma_s: float, N: int):
    """(sigma_i, a_i) for passes i = 1..N of the recursive filter."""
    sig = np.zeros(N)
    a = np.zeros(N)
    _load().orc_schedule(float(sigma_s), int(N), _ptr(sig), _ptr(a))
    return sig, a


def distances(I, sigma_s, sigma_r, norm=NORM_L1):
    """Domain-transform distances (dX, dY) of a (C, H, W) guide (Eq. 8-9)."""
    I = _f64(I)
    C, H, W = I.shape
    dX = np.empty((H, W))
    dY = np.empty((H, W))
    _load().orc_distances(C, H, W, _ptr(I), float(sigma_s), float(sigma_r), int(norm), _ptr(dX), _ptr(dY))
    return dX, dY


def causal(x, d, a):
    """Causal recurrence along a 1-D line (returns a new array)."""
    u = _f64(x).copy()
    d = _f64(d)
    _load().orc_causal(u.size, _ptr(u), 1, _ptr(d), 1, float(a))
    return u


def anticausal(x, d, a):
    """Anti-causal recurrence along a 1-D line (returns a new array)."""
    u = _f64(x).copy()
    d = _f64(d)
    _load().orc_anticausal(u.size, _ptr(u), 1, _ptr(d), 1, float(a))
    return u


def row_pass(u, dX, a):
    u = _f64(u).copy()
    dX = _f64(dX)
    H, W = u.shape
    _load().orc_row_pass(H, W, _ptr(u), _ptr(dX), float(a))
    return u


def col_pass(u, dY, a):
    u = _f64(u).copy()
    dY = _f64(dY)
    H, W = u.shape
    _load().orc_col_pass(H, W, _ptr(u), _ptr(dY), float(a))
    return u


def filter_d(dX, dY, a, src):
    """z_bar = A src for given distances and per-pass feedback coefficients a."""
    dX, dY, src = _f64(dX), _f64(dY), _f64(src)
    a = _f64(a)
    H, W = src.shape
    dst = np.empty((H, W))
    _load().orc_filter(H, W, _ptr(dX), _ptr(dY), a.size, _ptr(a), _ptr(src), _ptr(dst))
    return dst


def filter(I, src, sigma_s, sigma_r, passes=3, norm=NORM_L1):
    """Edge-aware mean of src under guide I (Eq. 10, recursive-filter kernel)."""
    dX, dY = distances(I, sigma_s, sigma_r, norm)
    _, a = schedule(sigma_s, passes)
    return filter_d(dX, dY, a, src)


def box_filter_d(dX, dY, sigma, src):
    """Box-kernel edge-aware mean (Eq. 10's printed kernel) for given distances and per-pass
    sigma_i (box radius sigma_i sqrt(3))."""
    dX, dY, src = _f64(dX), _f64(dY), _f64(src)
    sigma = _f64(sigma)
    H, W = src.shape
    dst = np.empty((H, W))
    _load().orc_box_filter(H, W, _ptr(dX), _ptr(dY), sigma.size, _ptr(sigma), _ptr(src), _ptr(dst))
    return dst


def box_filter(I, src, sigma_s, sigma_r, passes=3, norm=NORM_L1):
    """Box-kernel edge-aware mean of src under guide I."""
    dX, dY = distances(I, sigma_s, sigma_r, norm)
    sig, _ = schedule(sigma_s, passes)
    return box_filter_d(dX, dY, sig, src)


def confidence_d(dX, dY, a, t, sigma_c):
    """c = exp(-V / (2 sigma_c^2)), V = DT(t^2) - DT(t)^2 (Eq. 7) for given distances."""
    dX, dY, t = _f64(dX), _f64(dY), _f64(t)
    a = _f64(a)
    H, W = t.shape
    c = np.empty((H, W))
    _load().orc_confidence(H, W, _ptr(dX), _ptr(dY), a.size, _ptr(a), _ptr(t), float(sigma_c), _ptr(c))
    return c


def confidence(I, t, sigma_s, sigma_r, sigma_c, passes=3, norm=NORM_L1):
    """Confidence from the edge-aware variance of t under guide I (Eq. 7)."""
    dX, dY = distances(I, sigma_s, sigma_r, norm)
    _, a = schedule(sigma_s, passes)
    return confidence_d(dX, dY, a, t, sigma_c)


def support(dX, dY, sigma_s):
    """(S, S_flat): support sum_j W_ij of the unnormalised separable filter."""
    dX, dY = _f64(dX), _f64(dY)
    H, W = dX.shape
    S = np.empty((H, W))
    sf = ctypes.c_double(0.0)
    _load().orc_support(H, W, _ptr(dX), _ptr(dY), float(sigma_s), _ptr(S), ctypes.byref(sf))
    return S, sf.value


def solve_d(dX, dY, t, c, *, lam, sigma_s, step=0.99, iterations=10, passes=3, update=UPDATE_GD,
            conf_mode=CONF_PLAIN, z_init=None, checkpoints=False, kernel=KERNEL_RF, charbonnier_eps=0.0):
    """The solver on precomputed distances.  Returns z_K (and z_0..z_{K-1}).  kernel: the
    recursive filter (default) or the box kernel of Eq. 10.  charbonnier_eps > 0: the
    Charbonnier loss sqrt(r^2 + eps^2) on the target term (§4): the gradient step takes its
    slope, the fixed point of Eq. 4 its weight 1 / sqrt(r^2 + eps^2) at the current iterate."""
    dX, dY, t, c = _f64(dX), _f64(dY), _f64(t), _f64(c)
    z0 = None if z_init is None else _f64(z_init)
    H, W = t.shape
    z = np.empty((H, W))
    ck = np.empty((max(iterations, 1), H, W)) if checkpoints else None
    _load().orc_solve_kernel(H, W, _ptr(dX), _ptr(dY), _ptr(t), _ptr(c), _ptr(z0), float(lam), float(sigma_s),
                             float(step), int(iterations), int(passes), int(update), float(charbonnier_eps),
                             int(conf_mode), int(kernel), _ptr(z), _ptr(ck))
    if checkpoints:
        return z, ck[:iterations]
    return z


def solve(I, t, c, *, lam, sigma_s, sigma_r, step=0.99, iterations=10, passes=3, norm=NORM_L1,
          update=UPDATE_GD, conf_mode=CONF_PLAIN, z_init=None, checkpoints=False, kernel=KERNEL_RF,
          charbonnier_eps=0.0):
    """DTS solve on guide I (C, H, W) with target t and confidence c (H, W)."""
    dX, dY = distances(I, sigma_s, sigma_r, norm)
    return solve_d(dX, dY, t, c, lam=lam, sigma_s=sigma_s, step=step, iterations=iterations, passes=passes,
                   update=update, conf_mode=conf_mode, z_init=z_init, checkpoints=checkpoints, kernel=kernel,
                   charbonnier_eps=charbonnier_eps)


def solve_cg_d(dX, dY, t, c, *, lam, sigma_s, iterations=20, passes=3, z_init=None):
    """Conjugate gradients on Eq. 2 (lambda/2 |z - A z|^2 + sum c (z - t)^2) for given distances."""
    dX, dY, t, c = _f64(dX), _f64(dY), _f64(t), _f64(c)
    z0 = None if z_init is None else _f64(z_init)
    H, W = t.shape
    z = np.empty((H, W))
    _load().orc_solve_cg(H, W, _ptr(dX), _ptr(dY), _ptr(t), _ptr(c), _ptr(z0), float(lam), float(sigma_s),
                         int(iterations), int(passes), _ptr(z))
    return z


def solve_cg(I, t, c, *, lam, sigma_s, sigma_r, iterations=20, passes=3, norm=NORM_L1, z_init=None):
    """Conjugate gradients on Eq. 2 under guide I."""
    dX, dY = distances(I, sigma_s, sigma_r, norm)
    return solve_cg_d(dX, dY, t, c, lam=lam, sigma_s=sigma_s, iterations=iterations, passes=passes, z_init=z_init)


def filter_adjoint(dX, dY, a, src, gdst):
    """(A^T gdst, dXbar, dYbar) for the filter applied to src."""
    dX, dY, src, gdst, a = _f64(dX), _f64(dY), _f64(src), _f64(gdst), _f64(a)
    H, W = src.shape
    gsrc = np.empty((H, W))
    dXb = np.zeros((H, W))
    dYb = np.zeros((H, W))
    _load().orc_filter_adjoint(H, W, _ptr(dX), _ptr(dY), a.size, _ptr(a), _ptr(src), _ptr(gdst), _ptr(gsrc),
                               _ptr(dXb), _ptr(dYb))
    return gsrc, dXb, dYb


def distances_adjoint(I, sigma_s, sigma_r, dXbar, dYbar, norm=NORM_L1):
    I = _f64(I)
    C, H, W = I.shape
    dX, dY = distances(I, sigma_s, sigma_r, norm)
    gI = np.empty((C, H, W))
    _load().orc_distances_adjoint(C, H, W, _ptr(I), float(sigma_s), float(sigma_r), int(norm), _ptr(dX), _ptr(dY),
                                  _ptr(_f64(dXbar)), _ptr(_f64(dYbar)), _ptr(gI))
    return gI


def solve_backward(I, t, c, grad_z, *, lam, sigma_s, sigma_r, step=0.99, iterations=10, passes=3, norm=NORM_L1,
                   update=UPDATE_GD, conf_mode=CONF_PLAIN, z_init=None, charbonnier_eps=0.0):
    """Gradients of <grad_z, z_K> with respect to t, c, the guide and z_init.

    Returns a dict with keys ``t``, ``c``, ``guide`` and (when z_init is given)
    ``z_init``."""
    I, t, c, gz = _f64(I), _f64(t), _f64(c), _f64(grad_z)
    C, H, W = I.shape
    z0 = None if z_init is None else _f64(z_init)
    gt = np.empty((H, W))
    gc = np.empty((H, W))
    gI = np.empty((C, H, W))
    gz0 = np.empty((H, W)) if z0 is not None else None
    rc = _load().orc_solve_backward(C, H, W, _ptr(I), float(sigma_s), float(sigma_r), int(norm), _ptr(t), _ptr(c),
                                    _ptr(z0), float(lam), float(step), int(iterations), int(passes), int(update),
                                    float(charbonnier_eps), int(conf_mode), _ptr(gz), _ptr(gt), _ptr(gc), _ptr(gI),
                                    _ptr(gz0))
    if rc != 0:
        raise ValueError("oracle backward supports the PLAIN confidence mode only")
    out = {"t": gt, "c": gc, "guide": gI}
    if z0 is not None:
        out["z_init"] = gz0
    return out

"""Thin Python binding of libdts.so (the C ABI in include/dts.h).

Argument marshalling only: every step of the solver runs in the CUDA kernels
of the library.  Functions take CUDA torch tensors (device memory and the
current stream come from PyTorch) and keep the C entry-point names.  If the
library is missing or cannot be loaded, every call raises; there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
from typing import Optional

import torch

from . import build as _build

F32, BF16, F16 = 0, 1, 2
NORM_L1, NORM_L2 = 0, 1
UPDATE_GD, UPDATE_JACOBI, UPDATE_CG = 0, 1, 2
CONF_PLAIN, CONF_SUPPORT = 0, 1
KERNEL_RF, KERNEL_BOX = 0, 1

STATUS = {0: "DTS_OK", 1: "DTS_ERR_INVALID_ARG", 2: "DTS_ERR_UNSUPPORTED", 3: "DTS_ERR_WORKSPACE",
          4: "DTS_ERR_CUDA", 5: "DTS_ERR_TIMEOUT", 6: "DTS_ERR_NONFINITE"}

_TORCH_DTYPE = {torch.float32: F32, torch.bfloat16: BF16, torch.float16: F16}


class DTSError(RuntimeError):
    """A libdts call returned a non-zero status (``status``; names in ``STATUS``)."""

    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {STATUS.get(status, status)}")
        self.status = status


class CGuide(ctypes.Structure):
    """ctypes mirror of ``dts_guide`` (planar C x H x W guide: dtype, device pointer, strides)."""
    _fields_ = [("C", ctypes.c_int), ("H", ctypes.c_int), ("W", ctypes.c_int), ("dtype", ctypes.c_int),
                ("data", ctypes.c_void_p), ("ch_stride", ctypes.c_longlong), ("row_stride", ctypes.c_longlong)]


class CParams(ctypes.Structure):
    """ctypes mirror of ``dts_params`` (field order and types as in include/dts.h)."""
    _fields_ = [("lambda_", ctypes.c_float), ("sigma_s", ctypes.c_float), ("sigma_r", ctypes.c_float),
                ("step", ctypes.c_float), ("iterations", ctypes.c_int), ("passes", ctypes.c_int),
                ("norm", ctypes.c_int), ("update", ctypes.c_int), ("conf_mode", ctypes.c_int),
                ("dist_dtype", ctypes.c_int), ("save_checkpoints", ctypes.c_int), ("filter_kernel", ctypes.c_int),
                ("charbonnier_eps", ctypes.c_float)]


@dataclasses.dataclass
class Params:
    """Mirror of ``dts_params`` (see include/dts.h for the meaning of each field)."""
    lam: float = 1.0
    sigma_s: float = 8.0
    sigma_r: float = 0.2
    step: float = 0.99
    iterations: int = 10
    passes: int = 3
    norm: int = NORM_L1
    update: int = UPDATE_GD
    conf_mode: int = CONF_PLAIN
    dist_dtype: int = F32
    save_checkpoints: int = 0
    filter_kernel: int = KERNEL_RF
    charbonnier_eps: float = 0.0

    def c(self) -> CParams:
        """The ``dts_params`` struct these values describe."""
        return CParams(self.lam, self.sigma_s, self.sigma_r, self.step, self.iterations, self.passes, self.norm,
                       self.update, self.conf_mode, self.dist_dtype, self.save_checkpoints, self.filter_kernel,
                       self.charbonnier_eps)


_lib = None
EXPORTS = ("dts_status_string", "dts_version", "dts_workspace_size", "dts_domain_transform", "dts_filter",
           "dts_solve", "dts_solve_backward", "dts_last_status", "dts_profile", "dts_profile_read",
           "dts_kernel_name", "dts_solve_noalloc", "dts_noalloc_max_workspace", "dts_batched_workspace_size",
           "dts_solve_batched", "dts_debug_inject", "dts_autotune", "dts_autotune_export", "dts_autotune_import",
           "dts_autotune_batched",
           "dts_confidence")


def library_path() -> str:
    """Path of the in-tree libdts.so."""
    return _build.LIB


def load(build_if_missing: bool = True):
    """Open libdts.so (building it first if it is missing); raises on failure."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path) or not _build.up_to_date():
        if not build_if_missing:
            raise RuntimeError(f"libdts.so not built ({path}); run paper_1805_04590_gb300.build")
        _build.build()
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    vp, i, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
    lib.dts_status_string.argtypes = [i]
    lib.dts_status_string.restype = ctypes.c_char_p
    lib.dts_version.restype = ctypes.c_char_p
    lib.dts_workspace_size.argtypes = [P(CGuide), P(CParams), i]
    lib.dts_workspace_size.restype = sz
    lib.dts_domain_transform.argtypes = [P(CGuide), P(CParams), vp, vp, vp]
    lib.dts_filter.argtypes = [P(CGuide), P(CParams), vp, vp, vp, sz, vp]
    lib.dts_solve.argtypes = [P(CGuide), vp, i, vp, vp, P(CParams), vp, vp, sz, vp]
    lib.dts_solve_backward.argtypes = [P(CGuide), vp, i, vp, vp, P(CParams), vp, sz, vp, vp, vp, vp, vp, vp]
    lib.dts_confidence.argtypes = [P(CGuide), vp, i, P(CParams), ctypes.c_float, vp, vp, sz, vp]
    lib.dts_last_status.argtypes = [vp]
    lib.dts_solve_noalloc.argtypes = [P(CGuide), vp, i, vp, vp, P(CParams), vp, vp]
    lib.dts_batched_workspace_size.argtypes = [i, P(CGuide), P(CParams)]
    lib.dts_batched_workspace_size.restype = sz
    lib.dts_solve_batched.argtypes = [i, P(CGuide), P(vp), i, P(vp), P(CParams), P(vp), vp, sz, vp]
    lib.dts_autotune_batched.argtypes = [i, P(CGuide), P(vp), i, P(vp), P(CParams), P(vp), vp, sz, vp]
    lib.dts_debug_inject.argtypes = [i]
    lib.dts_autotune.argtypes = [P(CGuide), P(CParams), vp, sz, vp]
    lib.dts_autotune_export.argtypes = [ctypes.c_char_p, sz]
    lib.dts_autotune_import.argtypes = [ctypes.c_char_p]
    lib.dts_noalloc_max_workspace.restype = sz
    lib.dts_profile.argtypes = [i]
    lib.dts_profile_read.argtypes = [i, P(ctypes.c_int), P(ctypes.c_longlong), P(ctypes.c_int), P(ctypes.c_float)]
    lib.dts_kernel_name.argtypes = [i]
    lib.dts_kernel_name.restype = ctypes.c_char_p
    for name in ("dts_domain_transform", "dts_filter", "dts_solve", "dts_solve_backward", "dts_last_status",
                 "dts_confidence",
                 "dts_profile", "dts_profile_read", "dts_solve_noalloc", "dts_solve_batched", "dts_autotune_batched",
                 "dts_debug_inject",
                 "dts_autotune", "dts_autotune_export", "dts_autotune_import"):
        getattr(lib, name).restype = i
    _lib = lib
    return lib


def _check(status: int, what: str):
    if status != 0:
        raise DTSError(status, what)


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else t.data_ptr()


def _need_cuda(*ts):
    for t in ts:
        if t is not None and not t.is_cuda:
            raise ValueError("libdts takes CUDA tensors")


def guide_desc(guide: torch.Tensor) -> CGuide:
    """Describe a (C, H, W) or (H, W) CUDA tensor (row-contiguous) as a dts_guide."""
    if guide.dim() == 2:
        guide = guide.unsqueeze(0)
    if guide.dim() != 3 or guide.dtype not in _TORCH_DTYPE:
        raise ValueError("guide must be (C, H, W) float32/bfloat16/float16")
    if guide.stride(2) != 1:
        raise ValueError("guide rows must be contiguous")
    C, H, W = guide.shape
    return CGuide(C, H, W, _TORCH_DTYPE[guide.dtype], guide.data_ptr(), guide.stride(0), guide.stride(1))


def _dense(t: torch.Tensor, name: str, dtypes=(torch.float32,)):
    if t.dtype not in dtypes or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous {'/'.join(str(d) for d in dtypes)} tensor")


def workspace_size(guide: torch.Tensor, params: Params, with_backward: bool = False) -> int:
    """Bytes of workspace a solve (and, with_backward, its reverse mode) needs (dts_workspace_size)."""
    g = guide_desc(guide)
    p = params.c()
    return load().dts_workspace_size(ctypes.byref(g), ctypes.byref(p), int(with_backward))


def workspace(guide: torch.Tensor, params: Params, with_backward: bool = False) -> torch.Tensor:
    """A caller-owned workspace tensor of the size libdts asks for."""
    n = workspace_size(guide, params, with_backward)
    if n == 0:
        raise DTSError(1, "dts_workspace_size")
    return torch.empty(n, dtype=torch.uint8, device=guide.device)


def dts_domain_transform(guide: torch.Tensor, params: Params, stream=None):
    """(dX, dY) distance planes of the guide, dtype float32 or float16 per params.dist_dtype."""
    _need_cuda(guide)
    g = guide_desc(guide)
    H, W = g.H, g.W
    dt = torch.float16 if params.dist_dtype == F16 else torch.float32
    dX = torch.empty((H, W), dtype=dt, device=guide.device)
    dY = torch.empty((H, W), dtype=dt, device=guide.device)
    p = params.c()
    _check(load().dts_domain_transform(ctypes.byref(g), ctypes.byref(p), dX.data_ptr(), dY.data_ptr(),
                                       _stream(stream)), "dts_domain_transform")
    return dX, dY


def dts_filter(guide: torch.Tensor, src: torch.Tensor, params: Params, out: Optional[torch.Tensor] = None,
               ws: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """Edge-aware mean A src (H x W float32)."""
    _need_cuda(guide, src)
    _dense(src, "src")
    g = guide_desc(guide)
    out = torch.empty_like(src) if out is None else out
    ws = workspace(guide, params) if ws is None else ws
    p = params.c()
    _check(load().dts_filter(ctypes.byref(g), ctypes.byref(p), src.data_ptr(), out.data_ptr(), ws.data_ptr(),
                             ws.numel(), _stream(stream)), "dts_filter")
    return out


def dts_solve(guide: torch.Tensor, target: torch.Tensor, conf: torch.Tensor, params: Params,
              z_init: Optional[torch.Tensor] = None, out: Optional[torch.Tensor] = None,
              ws: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """The solver: returns z_K (H x W float32)."""
    _need_cuda(guide, target, conf, z_init)
    _dense(target, "target", tuple(_TORCH_DTYPE))
    _dense(conf, "conf")
    if z_init is not None:
        _dense(z_init, "z_init")
    g = guide_desc(guide)
    out = torch.empty(target.shape, dtype=torch.float32, device=target.device) if out is None else out
    ws = workspace(guide, params, bool(params.save_checkpoints)) if ws is None else ws
    p = params.c()
    _check(load().dts_solve(ctypes.byref(g), target.data_ptr(), _TORCH_DTYPE[target.dtype], conf.data_ptr(),
                            _ptr(z_init), ctypes.byref(p), out.data_ptr(), ws.data_ptr(), ws.numel(),
                            _stream(stream)), "dts_solve")
    return out


def dts_confidence(guide: torch.Tensor, target: torch.Tensor, params: Params, sigma_c: float,
                   out: Optional[torch.Tensor] = None, ws: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """Confidence exp(-V / (2 sigma_c^2)) from the edge-aware variance V = DT(t^2) - DT(t)^2 of the
    target (Eq. 7): H x W float32."""
    _need_cuda(guide, target)
    _dense(target, "target", tuple(_TORCH_DTYPE))
    g = guide_desc(guide)
    out = torch.empty(target.shape, dtype=torch.float32, device=target.device) if out is None else out
    p = dataclasses.replace(params, save_checkpoints=0)
    ws = workspace(guide, p) if ws is None else ws
    pc = p.c()
    _check(load().dts_confidence(ctypes.byref(g), target.data_ptr(), _TORCH_DTYPE[target.dtype], ctypes.byref(pc),
                                 float(sigma_c), out.data_ptr(), ws.data_ptr(), ws.numel(), _stream(stream)),
           "dts_confidence")
    return out


def batched_workspace(guides, params: Params) -> torch.Tensor:
    """Workspace tensor for dts_solve_batched over these guides."""
    arr = (CGuide * len(guides))(*[guide_desc(g) for g in guides])
    p = params.c()
    n = load().dts_batched_workspace_size(len(guides), arr, ctypes.byref(p))
    if n == 0:
        raise DTSError(1, "dts_batched_workspace_size")
    return torch.empty(n, dtype=torch.uint8, device=guides[0].device)


def dts_autotune(guide: torch.Tensor, params: Params, ws: Optional[torch.Tensor] = None, stream=None) -> None:
    """Time the candidate tile shapes for this guide's height and width and record the fastest."""
    g = guide_desc(guide)
    ws = workspace(guide, params) if ws is None else ws
    p = params.c()
    _check(load().dts_autotune(ctypes.byref(g), ctypes.byref(p), ws.data_ptr(), ws.numel(), _stream(stream)),
           "dts_autotune")


def autotune_export() -> str:
    """The tile shapes recorded by dts_autotune, as text ("row W items" / "col H items warps cluster")."""
    lib = load()
    n = lib.dts_autotune_export(None, 0)
    buf = ctypes.create_string_buffer(n)
    lib.dts_autotune_export(buf, n)
    return buf.value.decode()


def autotune_import(text: str) -> None:
    """Record tile shapes from text in the format of autotune_export."""
    _check(load().dts_autotune_import(text.encode()), "dts_autotune_import")


def autotune_save(path: str) -> None:
    """Write the recorded shapes to a JSON cache tagged with the device they were measured on."""
    import json
    dev = torch.cuda.get_device_properties(torch.cuda.current_device())
    with open(path, "w") as f:
        json.dump({"device": dev.name, "sm_count": dev.multi_processor_count, "shapes": autotune_export()}, f)


def autotune_load(path: str) -> bool:
    """Load a JSON cache written by autotune_save if it was measured on this kind of device."""
    import json
    with open(path) as f:
        d = json.load(f)
    dev = torch.cuda.get_device_properties(torch.cuda.current_device())
    if d.get("device") != dev.name or d.get("sm_count") != dev.multi_processor_count:
        return False
    autotune_import(d["shapes"])
    return True


def _batch_args(guides, targets, confs, params: Params, outs, ws):
    n = len(guides)
    if not (len(targets) == len(confs) == n) or n == 0:
        raise ValueError("guides, targets and confs must be non-empty lists of equal length")
    dt = targets[0].dtype
    for t, c in zip(targets, confs):
        _need_cuda(t, c)
        _dense(t, "target", (dt,))
        _dense(c, "conf")
    outs = [torch.empty(t.shape, dtype=torch.float32, device=t.device) for t in targets] if outs is None else outs
    garr = (CGuide * n)(*[guide_desc(g) for g in guides])
    tarr = (ctypes.c_void_p * n)(*[t.data_ptr() for t in targets])
    carr = (ctypes.c_void_p * n)(*[c.data_ptr() for c in confs])
    oarr = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
    ws = batched_workspace(guides, params) if ws is None else ws
    return n, garr, tarr, _TORCH_DTYPE[dt], carr, outs, oarr, ws


def dts_solve_batched(guides, targets, confs, params: Params, outs=None, ws: Optional[torch.Tensor] = None,
                      stream=None, autotune: bool = False):
    """Solves of uneven sizes (lists of CUDA tensors, same parameters) as one CUDA graph launch
    (one persistent kernel when the batch allows it).  With autotune=True the tile shapes of every
    distinct size are measured first, then the batch's two ways of running (dts_autotune_batched)."""
    if autotune:
        tuned = set()
        for g in guides:
            if tuple(g.shape) not in tuned:
                dts_autotune(g, params, stream=stream)
                tuned.add(tuple(g.shape))
    n, garr, tarr, tdt, carr, outs, oarr, ws = _batch_args(guides, targets, confs, params, outs, ws)
    p = params.c()
    lib = load()
    if autotune:
        _check(lib.dts_autotune_batched(n, garr, tarr, tdt, carr, ctypes.byref(p), oarr, ws.data_ptr(), ws.numel(),
                                        _stream(stream)), "dts_autotune_batched")
    _check(lib.dts_solve_batched(n, garr, tarr, tdt, carr, ctypes.byref(p), oarr, ws.data_ptr(), ws.numel(),
                                 _stream(stream)), "dts_solve_batched")
    return outs


def dts_autotune_batched(guides, targets, confs, params: Params, outs=None, ws: Optional[torch.Tensor] = None,
                         stream=None) -> str:
    """Times the batch's two ways of running (the persistent kernel, the graph of per-image launch
    sequences) and keeps the faster for batches of this composition; returns "persistent" or
    "graph"."""
    n, garr, tarr, tdt, carr, outs, oarr, ws = _batch_args(guides, targets, confs, params, outs, ws)
    p = params.c()
    _check(load().dts_autotune_batched(n, garr, tarr, tdt, carr, ctypes.byref(p), oarr, ws.data_ptr(), ws.numel(),
                                       _stream(stream)), "dts_autotune_batched")
    return "graph" if "batch 1" in autotune_export() else "persistent"


def dts_solve_noalloc(guide: torch.Tensor, target: torch.Tensor, conf: torch.Tensor, params: Params,
                      z_init: Optional[torch.Tensor] = None, out: Optional[torch.Tensor] = None,
                      stream=None) -> torch.Tensor:
    """dts_solve on the library's own scratch array, for callers that cannot allocate device
    memory for a workspace (sizes up to dts_noalloc_max_workspace() bytes of workspace; calls
    that overlap on the GPU race on the shared array)."""
    _need_cuda(guide, target, conf, z_init)
    _dense(target, "target", tuple(_TORCH_DTYPE))
    _dense(conf, "conf")
    g = guide_desc(guide)
    out = torch.empty(target.shape, dtype=torch.float32, device=target.device) if out is None else out
    p = params.c()
    _check(load().dts_solve_noalloc(ctypes.byref(g), target.data_ptr(), _TORCH_DTYPE[target.dtype],
                                    conf.data_ptr(), _ptr(z_init), ctypes.byref(p), out.data_ptr(),
                                    _stream(stream)), "dts_solve_noalloc")
    return out


def dts_solve_backward(guide: torch.Tensor, target: torch.Tensor, conf: torch.Tensor, params: Params,
                       ws: torch.Tensor, grad_z: torch.Tensor, z_init: Optional[torch.Tensor] = None,
                       need_guide: bool = True, stream=None, outs=None):
    """Gradients (target, conf, guide or None, z_init or None) given dL/dz_K, into new tensors or
    into ``outs`` = (target, conf, guide, z_init) gradient tensors (float32, dense; guide and
    z_init entries may be None when not wanted).

    Must follow ``dts_solve`` with ``save_checkpoints`` 1 or 2 on the same workspace."""
    _need_cuda(guide, target, conf, grad_z, z_init)
    _dense(grad_z, "grad_z")
    g = guide_desc(guide)
    dev = target.device
    if outs is not None:
        gt, gc, gg, gz0 = outs
        for x, name in ((gt, "target gradient"), (gc, "confidence gradient"), (gg, "guide gradient"),
                        (gz0, "z_init gradient")):
            if x is not None:
                _need_cuda(x)
                _dense(x, name)
        if z_init is None:
            gz0 = None
    else:
        gt = torch.empty(target.shape, dtype=torch.float32, device=dev)
        gc = torch.empty(target.shape, dtype=torch.float32, device=dev)
        gg = torch.empty((g.C, g.H, g.W), dtype=torch.float32, device=dev) if need_guide else None
        gz0 = torch.empty(target.shape, dtype=torch.float32, device=dev) if z_init is not None else None
    p = params.c()
    _check(load().dts_solve_backward(ctypes.byref(g), target.data_ptr(), _TORCH_DTYPE[target.dtype],
                                     conf.data_ptr(), _ptr(z_init), ctypes.byref(p), ws.data_ptr(), ws.numel(),
                                     grad_z.data_ptr(), gt.data_ptr(), gc.data_ptr(), _ptr(gg), _ptr(gz0),
                                     _stream(stream)), "dts_solve_backward")
    return gt, gc, gg, gz0


def dts_last_status(stream=None) -> int:
    """Synchronise the stream and return (and clear) the device-side status word."""
    return load().dts_last_status(_stream(stream))


def dts_profile(mode: int) -> None:
    """Per-launch event timing in libdts: 1 start (clearing earlier records), 2 resume, 0 stop."""
    _check(load().dts_profile(int(mode)), "dts_profile")


def dts_profile_read(max_records: int = 1 << 16):
    """Records [(kernel name, kernel id, pixels, flags, ms)] since dts_profile(True)."""
    lib = load()
    k = (ctypes.c_int * max_records)()
    px = (ctypes.c_longlong * max_records)()
    fl = (ctypes.c_int * max_records)()
    ms = (ctypes.c_float * max_records)()
    n = lib.dts_profile_read(max_records, k, px, fl, ms)
    if n < 0:
        raise DTSError(-n, "dts_profile_read")
    return [(lib.dts_kernel_name(k[i]).decode(), k[i], px[i], fl[i], ms[i]) for i in range(n)]


def version() -> str:
    """The library's version string."""
    return load().dts_version().decode()


class HostPipeline:
    """Solves step after step on inputs held in pinned host memory, overlapping copies with
    solves: the host-to-device copies of step i + 1 run on one copy stream and the
    device-to-host copies of step i - 1 on another while step i solves on the current stream
    (two device buffer sets, events between the streams).

    ``solve_fn(inputs, outputs)`` enqueues the solve on the current stream, reading the device
    tensors ``inputs`` (shaped like a step's host inputs) and writing ``outputs`` (shaped like a
    step's host outputs)."""

    def __init__(self, solve_fn, depth: int = 2, device=None):
        self.solve_fn = solve_fn
        self.depth = depth
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.h2d = torch.cuda.Stream(device=self.device)
        self.d2h = torch.cuda.Stream(device=self.device)
        self.copied = [torch.cuda.Event() for _ in range(depth)]
        self.solved = [torch.cuda.Event() for _ in range(depth)]
        self.read = [torch.cuda.Event() for _ in range(depth)]
        self.bufs = [None] * depth

    def _buffers(self, slot, hin, hout):
        key = [(tuple(x.shape), x.dtype) for x in hin + hout]
        if self.bufs[slot] is None or self.bufs[slot][0] != key:
            din = [torch.empty(x.shape, dtype=x.dtype, device=self.device) for x in hin]
            dout = [torch.empty(x.shape, dtype=x.dtype, device=self.device) for x in hout]
            self.bufs[slot] = (key, din, dout)
        return self.bufs[slot][1], self.bufs[slot][2]

    def run(self, host_inputs, host_outputs, start_event=None):
        """host_inputs / host_outputs: per step, lists of pinned CPU tensors.  Returns with every
        copy enqueued and the current stream waiting for the last one."""
        cur = torch.cuda.current_stream(self.device)
        if start_event is not None:
            self.h2d.wait_event(start_event)
        for i, (hin, hout) in enumerate(zip(host_inputs, host_outputs)):
            s = i % self.depth
            din, dout = self._buffers(s, list(hin), list(hout))
            self.h2d.wait_event(self.solved[s])  # the solve two steps back has read these inputs
            with torch.cuda.stream(self.h2d):
                for d, h in zip(din, hin):
                    d.copy_(h, non_blocking=True)
            self.copied[s].record(self.h2d)
            cur.wait_event(self.copied[s])
            cur.wait_event(self.read[s])  # the copy two steps back has read these outputs
            self.solve_fn(din, dout)
            self.solved[s].record(cur)
            self.d2h.wait_event(self.solved[s])
            with torch.cuda.stream(self.d2h):
                for h, d in zip(hout, dout):
                    h.copy_(d, non_blocking=True)
            self.read[s].record(self.d2h)
        cur.wait_stream(self.d2h)
        cur.wait_stream(self.h2d)


def backward_checkpoint_mode(guide: torch.Tensor, params: Params) -> int:
    """save_checkpoints for a solve that will be differentiated: 2 (keep every pass input,
    no recompute in the backward) when its workspace takes at most a quarter of the free
    device memory, else 1 (keep the iterates only)."""
    g = guide_desc(guide)
    p2 = dataclasses.replace(params, save_checkpoints=2).c()
    need = load().dts_workspace_size(ctypes.byref(g), ctypes.byref(p2), 1)
    free, _ = torch.cuda.mem_get_info(guide.device)
    return 2 if need and need <= free // 4 else 1


class DTSSolve(torch.autograd.Function):
    """z_K = dts_solve(guide, target, conf, z_init) with the hand-written CUDA backward.

    The forward keeps every pass input in its workspace when memory allows (else the
    iterates z_0 .. z_{K-1}, from which the backward recomputes the pass inputs); the
    backward (dts_solve_backward) runs the reversed recurrences, giving gradients for the
    target, the confidence, the guide (through the distances) and z_init."""

    @staticmethod
    def forward(ctx, guide, target, conf, z_init, params: Params):
        # what dts_solve_backward differentiates; refused here, before the workspace is allocated
        if params.update == UPDATE_CG or params.conf_mode != CONF_PLAIN or params.filter_kernel != KERNEL_RF:
            raise ValueError("DTSSolve: the backward supports the recursive-filter kernel, plain confidence and "
                             "the GD or Jacobi update only")
        p = dataclasses.replace(params, save_checkpoints=backward_checkpoint_mode(guide, params))
        ws = workspace(guide, p, with_backward=True)
        z = dts_solve(guide, target, conf, p, z_init=z_init, ws=ws)
        zi = z_init if z_init is not None else torch.empty(0, device=target.device)
        # the workspace holds the checkpoints: a saved tensor, kept while the graph is retained
        ctx.save_for_backward(guide, target, conf, zi, ws)
        ctx.params = p
        ctx.has_zinit = z_init is not None
        return z

    @staticmethod
    def backward(ctx, grad_z):
        guide, target, conf, zi, ws = ctx.saved_tensors
        gt, gc, gg, gz0 = dts_solve_backward(guide, target, conf, ctx.params, ws,
                                             grad_z.contiguous().float(),
                                             z_init=zi if ctx.has_zinit else None,
                                             need_guide=ctx.needs_input_grad[0])
        return (gg.to(guide.dtype).reshape(guide.shape) if ctx.needs_input_grad[0] else None,
                gt.to(target.dtype) if ctx.needs_input_grad[1] else None,
                gc if ctx.needs_input_grad[2] else None,
                gz0 if (ctx.has_zinit and ctx.needs_input_grad[3]) else None,
                None)


def solve(guide: torch.Tensor, target: torch.Tensor, conf: torch.Tensor, params: Params,
          z_init: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Differentiable DTS solve (autograd through the CUDA backward)."""
    return DTSSolve.apply(guide, target, conf, z_init, params)

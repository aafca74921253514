"""ctypes binding of libfunnel.so (include/funnel.h), same names as the C ABI.

Argument marshalling only: every step of the transform runs in the library's
CUDA kernels.  Tensors are torch CUDA tensors (device memory and streams come
from PyTorch); host-buffer calls take contiguous CPU tensors or numpy arrays.
There is no CPU fallback: if the library is not built, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Tuple

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
# FT_DEBUG=1 in the environment loads the bounds-checked build (ft_debug_flags)
LIB_PATH = os.path.join(PKG, "libfunnel_debug.so" if os.environ.get("FT_DEBUG") == "1" else "libfunnel.so")

FT_OK = 0
FT_ERR_INVALID_ARG = 1
FT_ERR_UNSUPPORTED_SIZE = 2
FT_ERR_OOM = 3
FT_ERR_CUDA = 4
FT_ERR_TIMEOUT = 5
FT_INTERP_LINEAR = 0
FT_INTERP_CUBIC = 1
FT_INTERP_FOURIER = 2
FT_MAX_LENGTH = 8192
FT_MAX_TOPK = 1024
INTERP_NAMES = {"linear": FT_INTERP_LINEAR, "cubic": FT_INTERP_CUBIC, "fourier": FT_INTERP_FOURIER}

EXPORTED = (
    "ft_plan_create", "ft_plan_destroy", "ft_forward", "ft_backward", "ft_peaks",
    "ft_detect_host", "ft_workspace_bytes", "ft_forward_launches", "ft_peaks_launches",
    "ft_status_string", "ft_last_error", "ft_profile_enable", "ft_profile_read", "ft_kernel_name",
    "ft_peaks_noalloc", "ft_abs_mse_grad", "ft_plan_create_space",
    "ft_plan_variant_count", "ft_plan_set_variant", "ft_plan_get_variant",
    "ft_batch_create", "ft_batch_destroy", "ft_batch_layout", "ft_batch_group_count",
    "ft_batch_group_info", "ft_batch_group_tuned_ms", "ft_batch_run", "ft_tc_dft64",
    "ft_plan_set_precision", "ft_plan_get_precision", "ft_plan_tc_errors", "ft_verify",
    "ft_abs_mse_backward", "ft_detect", "ft_detect_launches", "ft_detect_batches",
    "ft_plan_set_wait_cycles", "ft_plan_get_wait_cycles", "ft_plan_inject_alloc_failures",
    "ft_batch_config", "ft_batch_set_config", "ft_batch_tune_ms", "ft_batch_launches", "ft_fma_probe",
    "ft_debug_flags", "ft_debug_build",
)
FT_WAIT_CYCLES_DEFAULT = 4000000000
FT_PRECISION_FP32 = 0
FT_PRECISION_BF16X3 = 1
FT_PRECISION_FP16X3 = 2
FT_PRECISION_BF16X6 = 3
PRECISION_NAMES = {"fp32": FT_PRECISION_FP32, "bf16x3": FT_PRECISION_BF16X3, "fp16x3": FT_PRECISION_FP16X3,
                   "bf16x6": FT_PRECISION_BF16X6}
FT_BATCH_GRAPH = 1
FT_BATCH_TUNE = 2
FT_SPACE_REGULAR = 0
FT_SPACE_INVERSE = 1
SPACE_NAMES = {"regular": FT_SPACE_REGULAR, "inverse": FT_SPACE_INVERSE}
FT_NOALLOC_SCRATCH_BYTES = 16 << 20
FT_KERNEL_COUNT = 10


class FtPeak(ctypes.Structure):
    _fields_ = [("t", ctypes.c_int32), ("s", ctypes.c_int32), ("value", ctypes.c_float),
                ("k", ctypes.c_float), ("b", ctypes.c_float)]


PEAK_DTYPE = np.dtype([("t", np.int32), ("s", np.int32), ("value", np.float32),
                       ("k", np.float32), ("b", np.float32)])


class FunnelError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: status {status}" + (f" ({detail})" if detail else ""))


_lib: Optional[ctypes.CDLL] = None


def lib() -> ctypes.CDLL:
    """Load libfunnel.so (built by ``paper_1904_09409_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built; run `python -c \"import __graft_entry__ as g; "
                           "g.build()\"` first (there is no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    vp, ci, cf = ctypes.c_void_p, ctypes.c_int, ctypes.c_float
    L.ft_plan_create.argtypes = [ctypes.POINTER(vp), ci, ci, ci, ci, ci]
    L.ft_plan_create_space.argtypes = [ctypes.POINTER(vp), ci, ci, ci, ci, ci, ci]
    L.ft_plan_create_space.restype = ci
    L.ft_plan_destroy.argtypes = [vp]
    L.ft_forward.argtypes = [vp, vp, vp, ci, vp]
    L.ft_backward.argtypes = [vp, vp, vp, ci, vp]
    L.ft_peaks.argtypes = [vp, vp, ci, ci, cf, vp, vp, vp]
    L.ft_detect_host.argtypes = [vp, vp, ci, ci, cf, vp, vp, vp]
    L.ft_workspace_bytes.argtypes = [vp, ci]
    L.ft_workspace_bytes.restype = ctypes.c_size_t
    L.ft_forward_launches.argtypes = [vp, ci]
    L.ft_peaks_launches.argtypes = [vp, ci]
    L.ft_status_string.argtypes = [ci]
    L.ft_status_string.restype = ctypes.c_char_p
    L.ft_last_error.argtypes = []
    L.ft_last_error.restype = ctypes.c_char_p
    L.ft_profile_enable.argtypes = [vp, ci]
    L.ft_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32), ci]
    L.ft_kernel_name.argtypes = [ci]
    L.ft_kernel_name.restype = ctypes.c_char_p
    L.ft_peaks_noalloc.argtypes = [vp, ci, ci, ci, ci, cf, vp, vp, vp]
    L.ft_abs_mse_grad.argtypes = [vp, vp, vp, ci, cf, vp, vp, vp]
    L.ft_abs_mse_grad.restype = ci
    L.ft_plan_variant_count.argtypes = [vp]
    L.ft_plan_set_variant.argtypes = [vp, ci]
    L.ft_plan_get_variant.argtypes = [vp]
    L.ft_batch_create.argtypes = [ctypes.POINTER(vp), ci, vp, vp, ci, ctypes.c_char_p]
    L.ft_batch_destroy.argtypes = [vp]
    L.ft_batch_layout.argtypes = [vp, vp, vp, vp, vp]
    L.ft_batch_group_count.argtypes = [vp]
    L.ft_batch_group_info.argtypes = [vp, ci, vp]
    L.ft_batch_group_tuned_ms.argtypes = [vp, ci]
    L.ft_batch_group_tuned_ms.restype = cf
    L.ft_batch_run.argtypes = [vp, vp, vp, ci, cf, vp, vp, vp, ci]
    L.ft_tc_dft64.argtypes = [vp, vp, ci, ci, ci, vp, vp]
    L.ft_tc_dft64.restype = ci
    L.ft_plan_set_precision.argtypes = [vp, ci]
    L.ft_plan_set_precision.restype = ci
    L.ft_plan_get_precision.argtypes = [vp]
    L.ft_plan_get_precision.restype = ci
    L.ft_plan_tc_errors.argtypes = [vp, ctypes.POINTER(ctypes.c_uint32)]
    L.ft_plan_tc_errors.restype = ci
    L.ft_verify.argtypes = [vp, vp, vp, vp, ci, ci, ci, cf, ci, vp, vp, vp, vp]
    L.ft_verify.restype = ci
    L.ft_abs_mse_backward.argtypes = [vp, vp, vp, ci, cf, vp, vp, vp]
    L.ft_abs_mse_backward.restype = ci
    L.ft_detect.argtypes = [vp, vp, vp, ci, ci, cf, vp, vp, vp]
    L.ft_detect.restype = ci
    L.ft_detect_batches.argtypes = [vp, ctypes.POINTER(vp), ci, ci, vp, ci, cf, vp, vp, vp]
    L.ft_detect_batches.restype = ci
    L.ft_plan_set_wait_cycles.argtypes = [vp, ctypes.c_int64]
    L.ft_plan_set_wait_cycles.restype = ci
    L.ft_plan_get_wait_cycles.argtypes = [vp]
    L.ft_plan_get_wait_cycles.restype = ctypes.c_int64
    L.ft_plan_inject_alloc_failures.argtypes = [vp, ci]
    L.ft_plan_inject_alloc_failures.restype = ci
    L.ft_batch_config.argtypes = [vp, vp]
    L.ft_batch_config.restype = ci
    L.ft_batch_set_config.argtypes = [vp, ci, ci, ci]
    L.ft_batch_set_config.restype = ci
    L.ft_batch_tune_ms.argtypes = [vp, vp, ci]
    L.ft_batch_tune_ms.restype = ci
    L.ft_batch_launches.argtypes = [vp, ci]
    L.ft_batch_launches.restype = ci
    L.ft_fma_probe.argtypes = [vp, ci, ci, vp]
    L.ft_fma_probe.restype = ci
    L.ft_debug_flags.argtypes = [ctypes.POINTER(ctypes.c_uint32)]
    L.ft_debug_flags.restype = ci
    L.ft_debug_build.argtypes = []
    L.ft_debug_build.restype = ci
    L.ft_detect_launches.argtypes = [vp, ci, ci]
    L.ft_detect_launches.restype = ci
    for name in ("ft_plan_variant_count", "ft_plan_set_variant", "ft_plan_get_variant", "ft_batch_create",
                 "ft_batch_destroy", "ft_batch_layout", "ft_batch_group_count", "ft_batch_group_info",
                 "ft_batch_run"):
        getattr(L, name).restype = ci
    for name in ("ft_peaks_noalloc", "ft_profile_enable", "ft_profile_read", "ft_plan_create", "ft_plan_destroy", "ft_forward", "ft_backward", "ft_peaks",
                 "ft_detect_host", "ft_forward_launches", "ft_peaks_launches"):
        getattr(L, name).restype = ci
    _lib = L
    return L


def _check(status: int, where: str) -> None:
    if status != FT_OK:
        L = lib()
        text = L.ft_status_string(status).decode()
        detail = L.ft_last_error().decode() if status == FT_ERR_CUDA else ""
        raise FunnelError(status, where, text + (f"; {detail}" if detail else ""))


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dev_ptr(t, dtype_name: str, numel: int, what: str) -> int:
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what} must be a CUDA tensor")
    if t.dtype != getattr(torch, dtype_name) or not t.is_contiguous():
        raise TypeError(f"{what} must be a contiguous {dtype_name} tensor")
    if t.numel() < numel:
        raise ValueError(f"{what} holds {t.numel()} elements, needs {numel}")
    return t.data_ptr()


class Plan:
    """Owns an ft_plan handle; sizes as in ft_plan_create_space.  H, W are the
    image's sizes; the map is (n_intercept, n_slope), by default (H, W) for the
    regular space and (W, H) for the inverse space."""

    def __init__(self, H: int, W: int, n_slope: Optional[int] = None,
                 n_intercept: Optional[int] = None, interp="linear", space="regular"):
        self.H, self.W = int(H), int(W)
        self.space = SPACE_NAMES[space] if isinstance(space, str) else int(space)
        inv = self.space == FT_SPACE_INVERSE
        self.S = (self.H if inv else self.W) if n_slope is None else int(n_slope)
        self.Hp = (self.W if inv else self.H) if n_intercept is None else int(n_intercept)
        self.interp = INTERP_NAMES[interp] if isinstance(interp, str) else int(interp)
        self.handle = ft_plan_create_space(self.H, self.W, self.S, self.Hp, self.interp, self.space)

    def close(self):
        if self.handle:
            ft_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def map_shape(self) -> Tuple[int, int]:
        return self.Hp, self.S


# ------------------------------------------------------------ C-ABI functions
def ft_plan_create(H: int, W: int, n_slope: int, n_intercept: int, interp: int = FT_INTERP_LINEAR):
    h = ctypes.c_void_p()
    _check(lib().ft_plan_create(ctypes.byref(h), int(H), int(W), int(n_slope), int(n_intercept),
                                int(interp)), "ft_plan_create")
    return h


def ft_plan_create_space(H: int, W: int, n_slope: int, n_intercept: int, interp: int = FT_INTERP_LINEAR,
                         space: int = FT_SPACE_REGULAR):
    h = ctypes.c_void_p()
    _check(lib().ft_plan_create_space(ctypes.byref(h), int(H), int(W), int(n_slope), int(n_intercept),
                                      int(interp), int(space)), "ft_plan_create_space")
    return h


def ft_plan_destroy(plan) -> None:
    _check(lib().ft_plan_destroy(plan), "ft_plan_destroy")


def ft_forward(plan: Plan, img, out_map, batch: Optional[int] = None, stream=None) -> None:
    b = img.shape[0] if batch is None else int(batch)
    ip = _dev_ptr(img, "float32", b * plan.H * plan.W, "img")
    mp = _dev_ptr(out_map, "float32", b * plan.Hp * plan.S, "map")
    _check(lib().ft_forward(plan.handle, ip, mp, b, _stream_ptr(stream)), "ft_forward")


def ft_backward(plan: Plan, grad_map, grad_img, batch: Optional[int] = None, stream=None) -> None:
    b = grad_map.shape[0] if batch is None else int(batch)
    gp = _dev_ptr(grad_map, "float32", b * plan.Hp * plan.S, "grad_map")
    ip = _dev_ptr(grad_img, "float32", b * plan.H * plan.W, "grad_img")
    _check(lib().ft_backward(plan.handle, gp, ip, b, _stream_ptr(stream)), "ft_backward")


def ft_peaks(plan: Plan, fmap, top_k: int, threshold: float = float("-inf"), out=None, count=None,
             batch: Optional[int] = None, stream=None):
    """Returns (peaks, count): peaks a uint8 CUDA tensor holding [batch][top_k]
    ft_peak records (view with ``peaks_to_numpy``), count an int32 tensor."""
    import torch
    b = fmap.shape[0] if batch is None else int(batch)
    mp = _dev_ptr(fmap, "float32", b * plan.Hp * plan.S, "map")
    if out is None:
        out = torch.empty(b * top_k * PEAK_DTYPE.itemsize, dtype=torch.uint8, device=fmap.device)
    if count is None:
        count = torch.empty(b, dtype=torch.int32, device=fmap.device)
    op = _dev_ptr(out, "uint8", b * top_k * PEAK_DTYPE.itemsize, "out")
    cp = _dev_ptr(count, "int32", b, "count")
    _check(lib().ft_peaks(plan.handle, mp, b, int(top_k), float(threshold), op, cp,
                          _stream_ptr(stream)), "ft_peaks")
    return out, count


def ft_detect(plan: Plan, img, out_map, top_k: int, threshold: float = float("-inf"), out=None, count=None,
              batch: Optional[int] = None, stream=None):
    """ft_forward (img -> out_map) and ft_peaks of that map in one call (same
    results); returns (peaks, count) like ft_peaks."""
    import torch
    b = img.shape[0] if batch is None else int(batch)
    ip = _dev_ptr(img, "float32", b * plan.H * plan.W, "img")
    mp = _dev_ptr(out_map, "float32", b * plan.Hp * plan.S, "map")
    if out is None:
        out = torch.empty(b * top_k * PEAK_DTYPE.itemsize, dtype=torch.uint8, device=out_map.device)
    if count is None:
        count = torch.empty(b, dtype=torch.int32, device=out_map.device)
    op = _dev_ptr(out, "uint8", b * top_k * PEAK_DTYPE.itemsize, "out")
    cp = _dev_ptr(count, "int32", b, "count")
    _check(lib().ft_detect(plan.handle, ip, mp, b, int(top_k), float(threshold), op, cp, _stream_ptr(stream)),
           "ft_detect")
    return out, count


def ft_detect_batches(plan: Plan, imgs, out_map, top_k: int, threshold: float = float("-inf"), out=None,
                      count=None, stream=None):
    """ft_detect over the batches imgs[j] (CUDA float32 tensors of one shape
    (batch, H, W)) as one pipeline on the stream; out_map (batch maps) is shared
    scratch.  Returns (peaks, count): len(imgs) * batch * top_k records and
    len(imgs) * batch counts, batch j's first, equal to len(imgs) ft_detect
    calls."""
    import torch
    nb = len(imgs)
    b = imgs[0].shape[0] if nb else 0
    ptrs = (ctypes.c_void_p * max(nb, 1))()
    for j, t in enumerate(imgs):
        if t.shape[0] != b:
            raise ValueError("all batches must hold the same number of images")
        ptrs[j] = _dev_ptr(t, "float32", b * plan.H * plan.W, f"imgs[{j}]")
    mp = _dev_ptr(out_map, "float32", b * plan.Hp * plan.S, "map")
    dev = out_map.device
    if out is None:
        out = torch.empty(nb * b * top_k * PEAK_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    if count is None:
        count = torch.empty(nb * b, dtype=torch.int32, device=dev)
    op = _dev_ptr(out, "uint8", nb * b * top_k * PEAK_DTYPE.itemsize, "out")
    cp = _dev_ptr(count, "int32", nb * b, "count")
    _check(lib().ft_detect_batches(plan.handle, ptrs, nb, b, mp, int(top_k), float(threshold), op, cp,
                                   _stream_ptr(stream)), "ft_detect_batches")
    return out, count


def ft_verify(plan: Plan, img, peaks, count, top_k: int, half_width: int = 2, min_contrast: float = 0.1,
              min_length: int = 16, batch: Optional[int] = None, stream=None):
    """Line verification (Sec. 4.5) of the peaks ft_peaks wrote for this plan.
    img: the forward's input (batch, H, W) CUDA float32; peaks/count: ft_peaks'
    outputs.  Returns (profile [batch, top_k, 2h+1] float32, length
    [batch, top_k] int32, verdict [batch, top_k] int32: 1 line, 0 none, -1 no peak)."""
    import torch
    b = img.shape[0] if batch is None else int(batch)
    ip = _dev_ptr(img, "float32", b * plan.H * plan.W, "img")
    pp = _dev_ptr(peaks, "uint8", b * top_k * PEAK_DTYPE.itemsize, "peaks")
    cp = _dev_ptr(count, "int32", b, "count")
    nb = 2 * int(half_width) + 1
    prof = torch.empty((b, top_k, nb), dtype=torch.float32, device=img.device)
    length = torch.empty((b, top_k), dtype=torch.int32, device=img.device)
    verdict = torch.empty((b, top_k), dtype=torch.int32, device=img.device)
    _check(lib().ft_verify(plan.handle, ip, pp, cp, b, int(top_k), int(half_width), float(min_contrast),
                           int(min_length), prof.data_ptr(), length.data_ptr(), verdict.data_ptr(),
                           _stream_ptr(stream)), "ft_verify")
    return prof, length, verdict


def ft_peaks_noalloc(fmap, top_k: int, threshold: float = float("-inf"), out=None, count=None,
                     stream=None):
    """ft_peaks without a plan and without any device allocation inside the
    library (fixed scratch of FT_NOALLOC_SCRATCH_BYTES).  fmap: (batch, H', S)
    CUDA float32.  Returns (peaks, count) like ft_peaks; pass preallocated
    ``out``/``count`` to avoid allocations on the Python side too.  The call
    runs with fmap's device current (on ``stream``, by default that device's
    current stream); ``out`` and ``count`` must be on the same device."""
    import torch
    if not isinstance(fmap, torch.Tensor) or not fmap.is_cuda:
        raise TypeError("map must be a CUDA tensor")
    dev = fmap.device
    for t, what in ((out, "out"), (count, "count")):
        if t is not None and (not isinstance(t, torch.Tensor) or t.device != dev):
            raise TypeError(f"{what} must be a CUDA tensor on the map's device {dev}")
    b, Hp, S = (int(v) for v in fmap.shape)
    with torch.cuda.device(dev):
        mp = _dev_ptr(fmap, "float32", b * Hp * S, "map")
        if out is None:
            out = torch.empty(b * top_k * PEAK_DTYPE.itemsize, dtype=torch.uint8, device=dev)
        if count is None:
            count = torch.empty(b, dtype=torch.int32, device=dev)
        op = _dev_ptr(out, "uint8", b * top_k * PEAK_DTYPE.itemsize, "out")
        cp = _dev_ptr(count, "int32", b, "count")
        sp = torch.cuda.current_stream(dev).cuda_stream if stream is None else _stream_ptr(stream)
        st = lib().ft_peaks_noalloc(mp, Hp, S, b, int(top_k), float(threshold), op, cp, sp)
    if st == FT_ERR_UNSUPPORTED_SIZE:
        raise FunnelError(st, "ft_peaks_noalloc", ft_last_error())
    _check(st, "ft_peaks_noalloc")
    return out, count


def peaks_to_numpy(out, count, top_k: int):
    """Device peak records -> list (per image) of numpy structured arrays."""
    raw = out.cpu().numpy().view(PEAK_DTYPE).reshape(-1, top_k)
    cnt = count.cpu().numpy()
    return [raw[i, :cnt[i]] for i in range(raw.shape[0])]


def ft_detect_host(plan: Plan, img_host, top_k: int, threshold: float = float("-inf"),
                   out_host=None, count_host=None, stream=None):
    """End-to-end call on host buffers (pinned CPU tensors are fastest)."""
    import torch
    if isinstance(img_host, np.ndarray):
        img_host = torch.from_numpy(np.ascontiguousarray(img_host, dtype=np.float32))
    if img_host.is_cuda or img_host.dtype != torch.float32 or not img_host.is_contiguous():
        raise TypeError("img_host must be a contiguous float32 CPU tensor")
    b = img_host.shape[0]
    if out_host is None:
        out_host = torch.empty(b * top_k * PEAK_DTYPE.itemsize, dtype=torch.uint8)
    if count_host is None:
        count_host = torch.empty(b, dtype=torch.int32)
    _check(lib().ft_detect_host(plan.handle, img_host.data_ptr(), b, int(top_k), float(threshold),
                                out_host.data_ptr(), count_host.data_ptr(), _stream_ptr(stream)),
           "ft_detect_host")
    return out_host, count_host


def ft_abs_mse_grad(plan: Plan, fmap, target, scale: float, loss=None, grad=None, stream=None):
    """Per-image loss mean((|P| scale - T)^2) and the gradient of the batch mean
    (pass grad=False for the loss only).  Returns (loss, grad)."""
    import torch
    b = fmap.shape[0]
    n = b * plan.Hp * plan.S
    mp = _dev_ptr(fmap, "float32", n, "map")
    tp = _dev_ptr(target, "float32", n, "target")
    if loss is None:
        loss = torch.empty(b, dtype=torch.float32, device=fmap.device)
    if grad is None:
        grad = torch.empty_like(fmap)
    gp = _dev_ptr(grad, "float32", n, "grad") if grad is not False else None
    _check(lib().ft_abs_mse_grad(plan.handle, mp, tp, b, float(scale), _dev_ptr(loss, "float32", b, "loss"),
                                 gp, _stream_ptr(stream)), "ft_abs_mse_grad")
    return loss, (grad if grad is not False else None)


def ft_abs_mse_backward(plan: Plan, fmap, target, scale: float, loss=None, grad_img=None, stream=None):
    """The loss of ft_abs_mse_grad and its gradient with respect to the images
    in one call (the map gradient is never stored).  Returns (loss, grad_img)."""
    import torch
    b = fmap.shape[0]
    n = b * plan.Hp * plan.S
    mp = _dev_ptr(fmap, "float32", n, "map")
    tp = _dev_ptr(target, "float32", n, "target")
    if loss is None:
        loss = torch.empty(b, dtype=torch.float32, device=fmap.device)
    if grad_img is None:
        grad_img = torch.empty((b, plan.H, plan.W), dtype=torch.float32, device=fmap.device)
    gp = _dev_ptr(grad_img, "float32", b * plan.H * plan.W, "grad_img")
    _check(lib().ft_abs_mse_backward(plan.handle, mp, tp, b, float(scale), _dev_ptr(loss, "float32", b, "loss"),
                                     gp, _stream_ptr(stream)), "ft_abs_mse_backward")
    return loss, grad_img


def ft_workspace_bytes(plan: Plan, batch: int) -> int:
    return int(lib().ft_workspace_bytes(plan.handle, int(batch)))


def ft_forward_launches(plan: Plan, batch: int) -> int:
    return int(lib().ft_forward_launches(plan.handle, int(batch)))


def ft_peaks_launches(plan: Plan, batch: int) -> int:
    return int(lib().ft_peaks_launches(plan.handle, int(batch)))


def ft_detect_launches(plan: Plan, batch: int, top_k: int) -> int:
    return int(lib().ft_detect_launches(plan.handle, int(batch), int(top_k)))


def ft_profile_enable(plan: Plan, enable: bool = True) -> None:
    _check(lib().ft_profile_enable(plan.handle, int(bool(enable))), "ft_profile_enable")


def ft_profile_read(plan: Plan):
    """{kernel name: (total ms, launches)} of the launches recorded since the last read."""
    n = FT_KERNEL_COUNT
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_int32 * n)()
    _check(lib().ft_profile_read(plan.handle, ms, cnt, n), "ft_profile_read")
    return {ft_kernel_name(i): (float(ms[i]), int(cnt[i])) for i in range(n) if cnt[i]}


def ft_kernel_name(kernel_id: int) -> str:
    return lib().ft_kernel_name(int(kernel_id)).decode()


def ft_status_string(status: int) -> str:
    return lib().ft_status_string(int(status)).decode()


def ft_fma_probe(out, blocks: int, iters: int, stream=None) -> int:
    """FP32 FMA probe: returns the FLOPs of the call (time it with CUDA events)."""
    op = _dev_ptr(out, "float32", blocks * 256, "out")
    _check(lib().ft_fma_probe(op, int(blocks), int(iters), _stream_ptr(stream)), "ft_fma_probe")
    return blocks * 256 * iters * 16


def ft_debug_flags() -> int:
    """Index-check failures recorded by the debug build since the last call
    (FT_DBG_* bits; always 0 in the normal build).  Waits for the device."""
    v = ctypes.c_uint32(0)
    _check(lib().ft_debug_flags(ctypes.byref(v)), "ft_debug_flags")
    return int(v.value)


def ft_debug_build() -> bool:
    return bool(lib().ft_debug_build())


def ft_last_error() -> str:
    return lib().ft_last_error().decode()


def ft_tc_dft64(x, y, sign: int, precision, err, stream=None) -> None:
    """Batched 64-point DFTs on the tensor cores; x, y: complex64 CUDA tensors
    [nvec, 64]; err: int32 CUDA tensor of 1 element (bit 0 set on a wait timeout)."""
    import torch
    if x.dtype != torch.complex64 or y.dtype != torch.complex64 or not x.is_cuda or not y.is_cuda:
        raise TypeError("x and y must be complex64 CUDA tensors")
    if not (x.is_contiguous() and y.is_contiguous()) or x.shape[-1] != 64 or y.shape != x.shape:
        raise ValueError("x, y: contiguous [nvec, 64]")
    prec = PRECISION_NAMES[precision] if isinstance(precision, str) else int(precision)
    _check(lib().ft_tc_dft64(x.data_ptr(), y.data_ptr(), x.shape[0], int(sign), prec,
                             _dev_ptr(err, "int32", 1, "err"), _stream_ptr(stream)), "ft_tc_dft64")


def ft_plan_set_variant(plan: Plan, variant: int) -> None:
    _check(lib().ft_plan_set_variant(plan.handle, int(variant)), "ft_plan_set_variant")


def ft_plan_get_variant(plan: Plan) -> int:
    return int(lib().ft_plan_get_variant(plan.handle))


def ft_plan_set_precision(plan: Plan, precision) -> None:
    """Arithmetic of the length-4096 transforms: "fp32", "bf16x3", "fp16x3" or
    "bf16x6" (or the FT_PRECISION_* value)."""
    prec = PRECISION_NAMES[precision] if isinstance(precision, str) else int(precision)
    _check(lib().ft_plan_set_precision(plan.handle, prec), "ft_plan_set_precision")


def ft_plan_get_precision(plan: Plan) -> int:
    return int(lib().ft_plan_get_precision(plan.handle))


def ft_plan_tc_errors(plan: Plan) -> int:
    """Waits for the device, returns and clears the tensor-core error flags;
    raises FunnelError with status FT_ERR_TIMEOUT when a wait timed out."""
    v = ctypes.c_uint32(0)
    st = lib().ft_plan_tc_errors(plan.handle, ctypes.byref(v))
    if st == FT_ERR_TIMEOUT:
        raise FunnelError(st, "ft_plan_tc_errors", f"flags {int(v.value):#x}: {ft_last_error()}")
    _check(st, "ft_plan_tc_errors")
    return int(v.value)


def ft_plan_set_wait_cycles(plan: Plan, cycles: int) -> None:
    """Bound of the plan's tensor-core waits in SM cycles (0: give up at once)."""
    _check(lib().ft_plan_set_wait_cycles(plan.handle, int(cycles)), "ft_plan_set_wait_cycles")


def ft_plan_get_wait_cycles(plan: Plan) -> int:
    return int(lib().ft_plan_get_wait_cycles(plan.handle))


def ft_plan_inject_alloc_failures(plan: Plan, count: int) -> None:
    """The plan's next ``count`` device allocations fail with FT_ERR_OOM."""
    _check(lib().ft_plan_inject_alloc_failures(plan.handle, int(count)), "ft_plan_inject_alloc_failures")


class Batch:
    """A mixed-size batch (ft_batch_*): shapes is a list of (H, W); maps are
    n_intercept = H, n_slope = W.  Images, maps and peak rows live in one packed
    buffer each, in the batch's packed order (``order[j]`` = caller index)."""

    def __init__(self, shapes, interp="linear", tune_cache: Optional[str] = None):
        self.shapes = [(int(h), int(w)) for h, w in shapes]
        n = len(self.shapes)
        H = (ctypes.c_int32 * n)(*[h for h, _ in self.shapes])
        W = (ctypes.c_int32 * n)(*[w for _, w in self.shapes])
        h = ctypes.c_void_p()
        ip = INTERP_NAMES[interp] if isinstance(interp, str) else int(interp)
        _check(lib().ft_batch_create(ctypes.byref(h), n, ctypes.cast(H, ctypes.c_void_p),
                                     ctypes.cast(W, ctypes.c_void_p), ip,
                                     tune_cache.encode() if tune_cache else None), "ft_batch_create")
        self.handle = h
        self.n = n
        order = np.zeros(n, np.int32)
        ioff = np.zeros(n, np.int64)
        moff = np.zeros(n, np.int64)
        tot = np.zeros(2, np.int64)
        _check(lib().ft_batch_layout(h, order.ctypes.data, ioff.ctypes.data, moff.ctypes.data, tot.ctypes.data),
               "ft_batch_layout")
        self.order, self.img_off, self.map_off = order, ioff, moff
        self.img_total, self.map_total = int(tot[0]), int(tot[1])

    def groups(self):
        out = []
        info = np.zeros(5, np.int32)
        for g in range(int(lib().ft_batch_group_count(self.handle))):
            _check(lib().ft_batch_group_info(self.handle, g, info.ctypes.data), "ft_batch_group_info")
            out.append(dict(H=int(info[0]), W=int(info[1]), start=int(info[2]), count=int(info[3]),
                            variant=int(info[4]),
                            tuned_ms=float(lib().ft_batch_group_tuned_ms(self.handle, g))))
        return out

    def config(self):
        """The grouped kernels' configuration (ft_batch_config)."""
        info = np.zeros(6, np.int32)
        _check(lib().ft_batch_config(self.handle, info.ctypes.data), "ft_batch_config")
        return dict(grouped_images=int(info[0]), plan_groups=int(info[1]), r2c_threads=int(info[2]),
                    rows_threads=int(info[3]), c2r_threads=int(info[4]), launches=int(info[5]))

    def set_config(self, r2c_threads: int, rows_threads: int, c2r_threads: int) -> None:
        _check(lib().ft_batch_set_config(self.handle, int(r2c_threads), int(rows_threads), int(c2r_threads)),
               "ft_batch_set_config")

    def tune_ms(self):
        """{(r2c, rows, c2r threads): mean ms} measured by the autotuner (-1 before)."""
        ms = np.full(8, -1.0, np.float32)
        lib().ft_batch_tune_ms(self.handle, ms.ctypes.data, 8)
        return {((256, 512)[c >> 2 & 1], (128, 256)[c >> 1 & 1], (256, 512)[c & 1]): float(ms[c]) for c in range(8)}

    def launches(self, top_k: int = 1) -> int:
        return int(lib().ft_batch_launches(self.handle, int(top_k)))

    def pack(self, images):
        """List of (H, W) arrays in caller order -> packed float32 numpy buffer."""
        buf = np.empty(self.img_total, np.float32)
        for j, i in enumerate(self.order):
            h, w = self.shapes[i]
            buf[self.img_off[j]:self.img_off[j] + h * w] = np.asarray(images[i], np.float32).ravel()
        return buf

    def unpack_maps(self, maps):
        """Packed map buffer (numpy) -> list of (H, W) maps in caller order."""
        out = [None] * self.n
        for j, i in enumerate(self.order):
            h, w = self.shapes[i]
            out[i] = maps[self.map_off[j]:self.map_off[j] + h * w].reshape(h, w)
        return out

    def run(self, imgs, maps, top_k=0, threshold=float("-inf"), out=None, count=None, stream=None,
            graph=False, tune=False):
        ip = _dev_ptr(imgs, "float32", self.img_total, "imgs")
        mp = _dev_ptr(maps, "float32", self.map_total, "maps")
        op = _dev_ptr(out, "uint8", self.n * top_k * PEAK_DTYPE.itemsize, "out") if top_k else None
        cp = _dev_ptr(count, "int32", self.n, "count") if top_k else None
        flags = (FT_BATCH_GRAPH if graph else 0) | (FT_BATCH_TUNE if tune else 0)
        _check(lib().ft_batch_run(self.handle, ip, mp, int(top_k), float(threshold), op, cp,
                                  _stream_ptr(stream), flags), "ft_batch_run")

    def close(self):
        if self.handle:
            lib().ft_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# ------------------------------------------------------------ autograd wrapper
def funnel_transform(img, plan: Plan):
    """Differentiable forward: P = A img through ft_forward / ft_backward."""
    import torch

    class _Funnel(torch.autograd.Function):
        @staticmethod
        def forward(ctx, x):
            x = x.contiguous()
            out = torch.empty((x.shape[0], plan.Hp, plan.S), dtype=torch.float32, device=x.device)
            ft_forward(plan, x, out)
            return out

        @staticmethod
        def backward(ctx, g):
            g = g.contiguous()
            gi = torch.empty((g.shape[0], plan.H, plan.W), dtype=torch.float32, device=g.device)
            ft_backward(plan, g, gi)
            return gi

    return _Funnel.apply(img)

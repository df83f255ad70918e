"""GB300 local adaptive binarization (the Table 1 methods and the local quantile).

Thin ctypes binding over the C ABI declared in ``include/binarize.h``: every
function here only marshals torch tensors (device memory) and the current CUDA
stream into the C call of the same name; all arithmetic runs in the library's
CUDA kernels.  There is no CPU fallback: if ``libbinarize.so`` is missing,
every call raises.

Image tensors are uint8 CUDA tensors of shape (H, pitch) whose first W columns
hold the image (W defaults to the pitch).  Outputs are packed bits, shape
(H, out_pitch), bit (j & 7) of byte (j >> 3) = pixel j, 0 = foreground (I <= t).
"""
from __future__ import annotations

import ctypes
import os

from . import _build

__all__ = [
    "build", "library_path", "FP64", "FP32", "FP64_DIRECT", "SAUVOLA", "NIBLACK", "QUANTILE",
    "BinarizeError", "binarize_sauvola", "binarize_niblack", "binarize_quantile", "window_sums",
    "window_quantile", "binarize_precision_report", "last_fp64_fallbacks", "kernels_per_call", "Job",
    "binarize_batch",
    "binarize_batch_noalloc",
    "Server", "status_string",
    "WOLF", "FENG", "RAIS", "NICK", "PHANSALKAR", "binarize_wolf", "binarize_feng", "binarize_rais",
    "binarize_nick", "binarize_phansalkar", "global_stats", "binarize_precision_report_ext",
    "window_minmax", "binarize_bernsen", "haar_feature", "HAAR_FEATURES", "binarize_inplace",
    "inplace_scratch_bytes", "binarize_inplace_cols", "inplace_cols_scratch_bytes", "binarize_host", "binarize_host_multi",
    "autotune_window", "autotune_quantile", "autotune_batch", "tune_key", "tune_get", "tune_set",
    "tune_load", "tune_save", "tune_clear", "tune_window_plan", "bound_report", "use_library",
    "debug_status",
]

FP64, FP32, FP64_DIRECT = 0, 1, 2
SAUVOLA, NIBLACK, QUANTILE = 0, 1, 2
WOLF, FENG, RAIS, NICK, PHANSALKAR = 3, 4, 5, 6, 7
_PREC = {"fp64": FP64, "fp32": FP32, "fp64_direct": FP64_DIRECT, FP64: FP64, FP32: FP32,
         FP64_DIRECT: FP64_DIRECT}

_lib = None


class BinarizeError(RuntimeError):
    def __init__(self, fn: str, status: int):
        super().__init__(f"{fn}: {status_string(status)} (status {status})")
        self.status = status


def build(force: bool = False) -> str:
    """Compile the CUDA library in place (nvcc, sm_103a)."""
    global _lib
    path = _build.build(force=force)
    _lib = None
    return path


def library_path() -> str:
    return _build.LIB


class _JobC(ctypes.Structure):
    _fields_ = [("image", ctypes.c_void_p), ("out", ctypes.c_void_p), ("H", ctypes.c_int64),
                ("W", ctypes.c_int64), ("in_pitch", ctypes.c_int64), ("out_pitch", ctypes.c_int64),
                ("h", ctypes.c_int32), ("w", ctypes.c_int32), ("method", ctypes.c_int32),
                ("k", ctypes.c_double), ("R", ctypes.c_double), ("q_num", ctypes.c_int32),
                ("q_den", ctypes.c_int32), ("offset", ctypes.c_int32)]


class _HaarC(ctypes.Structure):
    _fields_ = [("n_row", ctypes.c_int32), ("n_col", ctypes.c_int32),
                ("row_len", ctypes.c_int32 * 4), ("row_wt", ctypes.c_int32 * 4),
                ("col_len", ctypes.c_int32 * 4), ("col_wt", ctypes.c_int32 * 4)]


_lib_path = None  # None: the normal build (libbinarize.so)


def use_library(debug: bool = False) -> str:
    """Route every following call to the normal library or to the
    bounds-checked debug build (built on first use); returns its path."""
    global _lib, _lib_path
    _lib_path = _build.build(debug=True) if debug else None
    _lib = None
    return _lib_path or _build.LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    path = _lib_path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first "
                           "(paper_1905_13038_gb300.build() or __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    P, i64, i32, f64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    st = ctypes.c_int
    sig = {
        "bz_status_string": ([st], ctypes.c_char_p),
        "binarize_sauvola": ([P, i64, i64, i64, i32, i32, f64, f64, P, i64, st, P], st),
        "binarize_niblack": ([P, i64, i64, i64, i32, i32, f64, P, i64, st, P], st),
        "binarize_quantile": ([P, i64, i64, i64, i32, i32, i32, i32, i32, P, i64, P], st),
        "window_sums": ([P, i64, i64, i64, i32, i32, P, P, P, P], st),
        "window_quantile": ([P, i64, i64, i64, i32, i32, i32, i32, P, P], st),
        "binarize_precision_report": ([i32, P, i64, i64, i64, i32, i32, f64, f64, P, P, P], st),
        "bz_last_fp64_fallbacks": ([P], i64),
        "bz_kernels_per_call": ([i64, i64, i32, i32, st], i32),
        "binarize_wolf": ([P, i64, i64, i64, i32, i32, f64, f64, P, i64, st, P], st),
        "binarize_feng": ([P, i64, i64, i64, i32, i32, f64, f64, f64, f64, f64, P, i64, st, P], st),
        "binarize_rais": ([P, i64, i64, i64, i32, i32, f64, P, i64, st, P], st),
        "binarize_nick": ([P, i64, i64, i64, i32, i32, f64, P, i64, st, P], st),
        "binarize_phansalkar": ([P, i64, i64, i64, i32, i32, f64, f64, f64, f64, P, i64, st, P], st),
        "global_stats": ([P, i64, i64, i64, P, P, P], st),
        "window_minmax": ([P, i64, i64, i64, i32, i32, P, P, P], st),
        "binarize_bernsen": ([P, i64, i64, i64, i32, i32, i32, P, i64, P], st),
        "haar_feature": ([P, i64, i64, i64, ctypes.POINTER(_HaarC), P, P], st),
        "binarize_inplace": ([i32, P, i64, i64, i64, i32, i32, f64, f64, i64, st, P], st),
        "binarize_host": ([i32, P, i64, i64, i64, i32, i32, f64, f64, P, i64, st, P], st),
        "binarize_host_multi": ([i32, P, i64, i64, i64, i32, P, P, f64, f64, P, i64, st, P], st),
        "bz_inplace_scratch_bytes": ([i64, i64, i32, i64], i64),
        "binarize_inplace_cols": ([i32, P, i64, i64, i64, i32, i32, f64, f64, i64, st, P], st),
        "bz_inplace_cols_scratch_bytes": ([i64, i64, i32, i64], i64),
        "binarize_precision_report_ext": ([i32, P, i64, i64, i64, i32, i32, P, P, P, P], st),
        "binarize_batch": ([ctypes.POINTER(_JobC), i32, st, P], st),
        "binarize_batch_noalloc": ([ctypes.POINTER(_JobC), i32, st, P], st),
        "bz_server_create": ([i64, i32, ctypes.POINTER(P)], st),
        "bz_server_submit": ([P, ctypes.POINTER(_JobC), st, ctypes.POINTER(ctypes.c_uint64)], st),
        "bz_server_wait": ([P, ctypes.c_uint64, i32], st),
        "bz_server_cancel": ([P, ctypes.c_uint64], st),
        "bz_server_destroy": ([P], st),
        "bz_debug_status": ([P, P, i32], i32),
        "binarize_bound_report": ([i32, P, i64, i64, i64, i32, i32, P, P, P], st),
        "bz_autotune_window": ([i32, P, i64, i64, i64, i32, i32, f64, f64, P, i64, st, P, P, P, P, P], st),
        "bz_autotune_quantile": ([P, i64, i64, i64, i32, i32, i32, i32, i32, P, i64, P, P, P], st),
        "bz_autotune_batch": ([ctypes.POINTER(_JobC), i32, st, P, P, P, P], st),
        "bz_tune_key": ([ctypes.c_char_p, ctypes.c_char_p, i32, i32, i32, i64, i64, ctypes.c_char_p, i32], i32),
        "bz_tune_get": ([ctypes.c_char_p, P, P, P, P], i32),
        "bz_tune_set": ([ctypes.c_char_p, i32, ctypes.c_float, i32, ctypes.c_float], i32),
        "bz_tune_load": ([ctypes.c_char_p], i32),
        "bz_tune_save": ([ctypes.c_char_p], i32),
        "bz_tune_clear": ([], None),
        "bz_tune_window_plan": ([ctypes.c_char_p, i32, i64, i64, i32, i32, i32, P], i32),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def status_string(status: int) -> str:
    return _load().bz_status_string(status).decode()


def _check(fn: str, status: int):
    if status != 0:
        raise BinarizeError(fn, status)


def _stream(stream):
    import torch
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _image(t, W):
    if t.dtype.itemsize != 1 or not t.is_cuda or t.dim() != 2 or t.stride(1) != 1:
        raise ValueError("image must be a 2-D uint8 CUDA tensor with unit column stride")
    H = t.shape[0]
    pitch = t.stride(0) if H > 1 else t.shape[1]
    W = t.shape[1] if W is None else W
    return t.data_ptr(), H, W, pitch


def _out(out, H, W, device):
    import torch
    if out is None:
        out = torch.empty((H, (W + 7) // 8), dtype=torch.uint8, device=device)
    if out.dtype.itemsize != 1 or not out.is_cuda or out.dim() != 2 or out.stride(1) != 1:
        raise ValueError("out must be a 2-D uint8 CUDA tensor with unit column stride")
    pitch = out.stride(0) if out.shape[0] > 1 else out.shape[1]
    return out, pitch


def binarize_sauvola(image, h: int, w: int, k: float = 0.5, R: float = 128.0, out=None,
                     precision="fp64", W: int | None = None, stream=None):
    ptr, H, W, pitch = _image(image, W)
    out, op = _out(out, H, W, image.device)
    _check("binarize_sauvola", _load().binarize_sauvola(ptr, H, W, pitch, h, w, k, R, out.data_ptr(), op,
                                                        _PREC[precision], _stream(stream)))
    return out


def binarize_niblack(image, h: int, w: int, k: float = -0.2, out=None, precision="fp64",
                     W: int | None = None, stream=None):
    ptr, H, W, pitch = _image(image, W)
    out, op = _out(out, H, W, image.device)
    _check("binarize_niblack", _load().binarize_niblack(ptr, H, W, pitch, h, w, k, out.data_ptr(), op,
                                                        _PREC[precision], _stream(stream)))
    return out


def binarize_quantile(image, h: int, w: int, q_num: int = 1, q_den: int = 2, offset: int = 8,
                      out=None, W: int | None = None, stream=None):
    ptr, H, W, pitch = _image(image, W)
    out, op = _out(out, H, W, image.device)
    _check("binarize_quantile", _load().binarize_quantile(ptr, H, W, pitch, h, w, q_num, q_den, offset,
                                                          out.data_ptr(), op, _stream(stream)))
    return out


def window_sums(image, h: int, w: int, W: int | None = None, stream=None):
    """(S1 int32-view of uint32, S2 int64-view of uint64, n) CUDA tensors (H, W)."""
    import torch
    ptr, H, W, pitch = _image(image, W)
    S1 = torch.empty((H, W), dtype=torch.int32, device=image.device)
    S2 = torch.empty((H, W), dtype=torch.int64, device=image.device)
    n = torch.empty((H, W), dtype=torch.int32, device=image.device)
    _check("window_sums", _load().window_sums(ptr, H, W, pitch, h, w, S1.data_ptr(), S2.data_ptr(),
                                              n.data_ptr(), _stream(stream)))
    return S1, S2, n


def window_quantile(image, h: int, w: int, q_num: int = 1, q_den: int = 2, W: int | None = None,
                    stream=None):
    import torch
    ptr, H, W, pitch = _image(image, W)
    Q = torch.empty((H, W), dtype=torch.uint8, device=image.device)
    _check("window_quantile", _load().window_quantile(ptr, H, W, pitch, h, w, q_num, q_den, Q.data_ptr(),
                                                      _stream(stream)))
    return Q


def binarize_precision_report(method: int, image, h: int, w: int, k: float, R: float = 128.0,
                              W: int | None = None, stream=None):
    """(flips, max |t32 - t64|) as Python numbers (synchronises the stream)."""
    import torch
    ptr, H, W, pitch = _image(image, W)
    flips = torch.zeros(1, dtype=torch.int64, device=image.device)
    maxdt = torch.zeros(1, dtype=torch.float64, device=image.device)
    torch.cuda.synchronize(image.device)  # the zeros are in place before `stream` runs
    _check("binarize_precision_report",
           _load().binarize_precision_report(method, ptr, H, W, pitch, h, w, k, R, flips.data_ptr(),
                                             maxdt.data_ptr(), _stream(stream)))
    torch.cuda.synchronize(image.device)  # ... and the report is complete before reading
    return int(flips.item()), float(maxdt.item())


def binarize_wolf(image, h: int, w: int, k: float = 0.5, R: float = 128.0, out=None,
                  precision="fp64", W: int | None = None, stream=None):
    """Wolf et al. (Table 1): t = m - k (m - L)(1 - s/R), L the global minimum."""
    ptr, H, W, pitch = _image(image, W)
    out, op = _out(out, H, W, image.device)
    _check("binarize_wolf", _load().binarize_wolf(ptr, H, W, pitch, h, w, k, R, out.data_ptr(), op,
                                                  _PREC[precision], _stream(stream)))
    return out


def binarize_feng(image, h: int, w: int, alpha1: float = 0.88, k1: float = 0.25, k2: float = 0.04,
                  gamma: float = 2.0, R: float = 128.0, out=None, precision="fp64",
                  W: int | None = None, stream=None):
    """Feng et al. in the Table 1 form
    t = alpha1 m + k1 (s/R)^(1+gamma) (m - L) + k2 (s/R)^gamma L."""
    ptr, H, W, pitch = _image(image, W)
    out, op = _out(out, H, W, image.device)
    _check("binarize_feng", _load().binarize_feng(ptr, H, W, pitch, h, w, alpha1, k1, k2, gamma, R,
                                                  out.data_ptr(), op, _PREC[precision], _stream(stream)))
    return out


def binarize_rais(image, h: int, w: int, k: float = 0.3, out=None, precision="fp64",
                  W: int | None = None, stream=None):
    """Rais et al. (Table 1): t = m + k (m s - M S) / max(m s, M S) s."""
    ptr, H, W, pitch = _image(image, W)
    out, op = _out(out, H, W, image.device)
    _check("binarize_rais", _load().binarize_rais(ptr, H, W, pitch, h, w, k, out.data_ptr(), op,
                                                  _PREC[precision], _stream(stream)))
    return out


def binarize_nick(image, h: int, w: int, k: float = -0.1, out=None, precision="fp64",
                  W: int | None = None, stream=None):
    """Khurshid et al. (NICK, Table 1): t = m + k sqrt(s^2 + m^2 (n - 1)/n)."""
    ptr, H, W, pitch = _image(image, W)
    out, op = _out(out, H, W, image.device)
    _check("binarize_nick", _load().binarize_nick(ptr, H, W, pitch, h, w, k, out.data_ptr(), op,
                                                  _PREC[precision], _stream(stream)))
    return out


def binarize_phansalkar(image, h: int, w: int, k: float = 0.25, R: float = 127.5, p: float = 2.0,
                        q: float = 10.0 / 255.0, out=None, precision="fp64", W: int | None = None,
                        stream=None):
    """Phansalkar et al. (Table 1): t = m (1 + p exp(-q m) + k (s/R - 1)) on gray
    levels 0..255 (the published normalised p = 2, q = 10, R = 0.5 are the defaults)."""
    ptr, H, W, pitch = _image(image, W)
    out, op = _out(out, H, W, image.device)
    _check("binarize_phansalkar", _load().binarize_phansalkar(ptr, H, W, pitch, h, w, k, R, p, q,
                                                              out.data_ptr(), op, _PREC[precision],
                                                              _stream(stream)))
    return out


def global_stats(image, W: int | None = None, stream=None):
    """((L, M, S) float64 CUDA tensor, (sum, sumsq, N) int64 CUDA tensor)."""
    import torch
    ptr, H, W, pitch = _image(image, W)
    stats = torch.empty(3, dtype=torch.float64, device=image.device)
    sums = torch.empty(3, dtype=torch.int64, device=image.device)
    _check("global_stats", _load().global_stats(ptr, H, W, pitch, stats.data_ptr(), sums.data_ptr(),
                                                _stream(stream)))
    return stats, sums


def binarize_precision_report_ext(method: int, image, h: int, w: int, params, W: int | None = None,
                                  stream=None):
    """(flips, max |t32 - t64|) for any Table 1 method; params = {k, R, alpha1,
    k1, k2, gamma, p, q} (8 floats)."""
    import torch
    ptr, H, W, pitch = _image(image, W)
    prm = (ctypes.c_double * 8)(*[float(x) for x in params])
    flips = torch.zeros(1, dtype=torch.int64, device=image.device)
    maxdt = torch.zeros(1, dtype=torch.float64, device=image.device)
    torch.cuda.synchronize(image.device)
    _check("binarize_precision_report_ext",
           _load().binarize_precision_report_ext(method, ptr, H, W, pitch, h, w, prm, flips.data_ptr(),
                                                 maxdt.data_ptr(), _stream(stream)))
    torch.cuda.synchronize(image.device)
    return int(flips.item()), float(maxdt.item())


def window_minmax(image, h: int, w: int, W: int | None = None, stream=None):
    """(min, max) uint8 CUDA tensors (H, W) of the clipped window."""
    import torch
    ptr, H, W, pitch = _image(image, W)
    mn = torch.empty((H, W), dtype=torch.uint8, device=image.device)
    mx = torch.empty((H, W), dtype=torch.uint8, device=image.device)
    _check("window_minmax", _load().window_minmax(ptr, H, W, pitch, h, w, mn.data_ptr(), mx.data_ptr(),
                                                  _stream(stream)))
    return mn, mx


def binarize_bernsen(image, h: int, w: int, contrast_limit: int = 15, out=None, W: int | None = None,
                     stream=None):
    """Bernsen: midrange threshold where the window's contrast reaches the
    limit, else the whole window is one class (dark iff its midrange <= 127.5)."""
    ptr, H, W, pitch = _image(image, W)
    out, op = _out(out, H, W, image.device)
    _check("binarize_bernsen", _load().binarize_bernsen(ptr, H, W, pitch, h, w, contrast_limit,
                                                        out.data_ptr(), op, _stream(stream)))
    return out


# Viola and Jones's feature shapes as (row segments, column segments) of an
# h x w window: two rectangles (edge), three (line), four (diagonal).
HAAR_FEATURES = {
    "edge_h": lambda h, w: ([(h, 1)], [(w // 2, 1), (w - w // 2, -1)]),
    "edge_v": lambda h, w: ([(h // 2, 1), (h - h // 2, -1)], [(w, 1)]),
    "line_h": lambda h, w: ([(h, 1)], [(w // 3, -1), (w - 2 * (w // 3), 2), (w // 3, -1)]),
    "line_v": lambda h, w: ([(h // 3, -1), (h - 2 * (h // 3), 2), (h // 3, -1)], [(w, 1)]),
    "diag": lambda h, w: ([(h // 2, 1), (h - h // 2, -1)], [(w // 2, 1), (w - w // 2, -1)]),
}


def haar_feature(image, rows, cols, out=None, W: int | None = None, stream=None):
    """int32 CUDA tensor (H, W): sum over the window of f(a) g(b) I, rows / cols
    = lists of (length, weight) segments (see HAAR_FEATURES for presets)."""
    import torch
    ptr, H, W, pitch = _image(image, W)
    if out is None:
        out = torch.empty((H, W), dtype=torch.int32, device=image.device)
    spec = _HaarC()
    spec.n_row, spec.n_col = len(rows), len(cols)
    if not (1 <= len(rows) <= 4 and 1 <= len(cols) <= 4):
        raise ValueError("1 to 4 segments per direction")
    for k, (n, wt) in enumerate(rows):
        spec.row_len[k], spec.row_wt[k] = n, wt
    for k, (n, wt) in enumerate(cols):
        spec.col_len[k], spec.col_wt[k] = n, wt
    _check("haar_feature", _load().haar_feature(ptr, H, W, pitch, ctypes.byref(spec), out.data_ptr(),
                                                _stream(stream)))
    return out


def binarize_inplace(method: int, image, h: int, w: int, k: float = 0.5, R: float = 128.0,
                     band_rows: int = 0, precision="fp64", W: int | None = None, stream=None):
    """Sauvola / Niblack written over `image`: each row then starts with its
    ceil(W/8) packed output bytes.  Returns the image tensor."""
    ptr, H, W, pitch = _image(image, W)
    _check("binarize_inplace", _load().binarize_inplace(method, ptr, H, W, pitch, h, w, k, R, band_rows,
                                                        _PREC[precision], _stream(stream)))
    return image


def binarize_inplace_cols(method: int, image, h: int, w: int, k: float = 0.5, R: float = 128.0,
                          band_cols: int = 0, precision="fp64", W: int | None = None, stream=None):
    """binarize_inplace with the axes exchanged: column bands over all rows,
    scratch proportional to H.  Returns the image tensor."""
    ptr, H, W, pitch = _image(image, W)
    _check("binarize_inplace_cols", _load().binarize_inplace_cols(method, ptr, H, W, pitch, h, w, k, R,
                                                                  band_cols, _PREC[precision],
                                                                  _stream(stream)))
    return image


def binarize_host(method: int, image, h: int, w: int, k: float = 0.5, R: float = 128.0, out=None,
                  precision="fp64", W: int | None = None, stream=None, sync: bool = True):
    """Sauvola / Niblack from host memory: `image` is a 2-D uint8 CPU tensor
    (pinned for asynchronous copies) whose first W columns hold the image;
    returns the packed output as a CPU uint8 tensor (H, ceil(W/8)).  With
    sync=False the call only enqueues: synchronise `stream` before reading."""
    import torch
    if image.is_cuda or image.dtype != torch.uint8 or image.dim() != 2 or image.stride(1) != 1:
        raise ValueError("image must be a 2-D uint8 CPU tensor with unit column stride")
    H = image.shape[0]
    pitch = image.stride(0) if H > 1 else image.shape[1]
    W = image.shape[1] if W is None else W
    if out is None:
        out = torch.empty((H, (W + 7) // 8), dtype=torch.uint8, pin_memory=image.is_pinned())
    op = out.stride(0) if out.shape[0] > 1 else out.shape[1]
    s = _stream(stream)
    _check("binarize_host", _load().binarize_host(method, image.data_ptr(), H, W, pitch, h, w, k, R,
                                                  out.data_ptr(), op, _PREC[precision], s))
    if sync:
        torch.cuda.Stream(stream_ptr=s.value).synchronize() if s.value else torch.cuda.synchronize()
    return out


def binarize_host_multi(method: int, image, windows, k: float = 0.5, R: float = 128.0, outs=None,
                        precision="fp64", W: int | None = None, stream=None, sync: bool = True):
    """binarize_host for several window sizes of one image: one upload, one
    packed output per (h, w) in `windows` (CPU uint8 tensors (H, ceil(W/8)),
    returned as a list).  With sync=False the call only enqueues."""
    import torch
    if image.is_cuda or image.dtype != torch.uint8 or image.dim() != 2 or image.stride(1) != 1:
        raise ValueError("image must be a 2-D uint8 CPU tensor with unit column stride")
    H = image.shape[0]
    pitch = image.stride(0) if H > 1 else image.shape[1]
    W = image.shape[1] if W is None else W
    n = len(windows)
    if outs is None:
        outs = [torch.empty((H, (W + 7) // 8), dtype=torch.uint8, pin_memory=image.is_pinned())
                for _ in range(n)]
    if len(outs) != n or n == 0:
        raise ValueError("one output per window")
    op = outs[0].stride(0) if outs[0].shape[0] > 1 else outs[0].shape[1]
    if any((o.stride(0) if o.shape[0] > 1 else o.shape[1]) != op for o in outs):
        raise ValueError("outputs must share one row pitch")
    hs = (ctypes.c_int32 * n)(*[int(h) for h, _ in windows])
    ws = (ctypes.c_int32 * n)(*[int(w) for _, w in windows])
    ptrs = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
    s = _stream(stream)
    _check("binarize_host_multi", _load().binarize_host_multi(method, image.data_ptr(), H, W, pitch, n, hs, ws,
                                                              k, R, ptrs, op, _PREC[precision], s))
    if sync:
        torch.cuda.Stream(stream_ptr=s.value).synchronize() if s.value else torch.cuda.synchronize()
    return outs


def inplace_scratch_bytes(H: int, W: int, h: int, band_rows: int = 0) -> int:
    return int(_load().bz_inplace_scratch_bytes(H, W, h, band_rows))


def inplace_cols_scratch_bytes(H: int, W: int, w: int, band_cols: int = 0) -> int:
    return int(_load().bz_inplace_cols_scratch_bytes(H, W, w, band_cols))


def last_fp64_fallbacks(stream=None) -> int:
    return int(_load().bz_last_fp64_fallbacks(_stream(stream)))


def kernels_per_call(H: int, W: int, h: int, w: int, precision="fp64") -> int:
    """Kernels one binarize_sauvola / binarize_niblack call launches on the
    current device for this geometry (window kernel plus stripe pre-pass)."""
    return int(_load().bz_kernels_per_call(H, W, h, w, _PREC[precision]))


class Job:
    """One image of a batch or a served request (tensors stay owned by the caller).
    inplace=True (served Sauvola / Niblack requests only): the packed result
    replaces the first ceil(W/8) bytes of each image row (out is the image)."""

    def __init__(self, image, method: int, h: int, w: int, k: float = 0.5, R: float = 128.0,
                 q_num: int = 1, q_den: int = 2, offset: int = 8, out=None, W: int | None = None,
                 inplace: bool = False):
        ptr, H, W, pitch = _image(image, W)
        self.image = image
        if inplace:
            self.out, self.out_pitch = image, pitch
        else:
            self.out, self.out_pitch = _out(out, H, W, image.device)
        self.c = _JobC(ptr, self.out.data_ptr(), H, W, pitch, self.out_pitch, h, w, method, k, R,
                       q_num, q_den, offset)


def binarize_batch(jobs, precision="fp64", stream=None):
    arr = (_JobC * len(jobs))(*[j.c for j in jobs])
    _check("binarize_batch", _load().binarize_batch(arr, len(jobs), _PREC[precision], _stream(stream)))
    return [j.out for j in jobs]


def binarize_batch_noalloc(jobs, precision="fp64", stream=None):
    """Same results as binarize_batch without any device allocation (at most
    512 jobs per call; calls that overlap on the GPU race on the shared work
    list)."""
    arr = (_JobC * len(jobs))(*[j.c for j in jobs])
    _check("binarize_batch_noalloc",
           _load().binarize_batch_noalloc(arr, len(jobs), _PREC[precision], _stream(stream)))
    return [j.out for j in jobs]


class Server:
    """Continuous-batching server (bz_server_*)."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int = 64):
        self._h = ctypes.c_void_p()
        _check("bz_server_create", _load().bz_server_create(hbm_budget_bytes, max_slots,
                                                            ctypes.byref(self._h)))
        self._jobs = {}

    def submit(self, job: Job, precision="fp64") -> int:
        t = ctypes.c_uint64()
        _check("bz_server_submit", _load().bz_server_submit(self._h, ctypes.byref(job.c),
                                                            _PREC[precision], ctypes.byref(t)))
        self._jobs[t.value] = job
        return t.value

    def wait(self, ticket: int, timeout_ms: int = -1) -> int:
        st = _load().bz_server_wait(self._h, ticket, timeout_ms)
        if st != 6:  # after BZ_ETIMEOUT a running request still uses its buffers
            self._jobs.pop(ticket, None)
        return st

    def cancel(self, ticket: int) -> int:
        return _load().bz_server_cancel(self._h, ticket)

    def close(self):
        if self._h:
            _check("bz_server_destroy", _load().bz_server_destroy(self._h))
            self._h = ctypes.c_void_p()
            self._jobs.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def debug_status(reset: bool = True):
    """(status bits, first offending address) of the bounds-checked build, or
    None from the normal build (bz_debug_status)."""
    st, addr = ctypes.c_uint32(), ctypes.c_uint64()
    r = _load().bz_debug_status(ctypes.byref(st), ctypes.byref(addr), 1 if reset else 0)
    if r < 0:
        raise RuntimeError("bz_debug_status failed")
    return None if r == 1 else (st.value, addr.value)


def bound_report(method: int, image, h: int, w: int, params, W: int | None = None, stream=None) -> float:
    """max over pixels of |t32 - t64| / certified bound (binarize_bound_report)."""
    import torch
    ptr, H, W, pitch = _image(image, W)
    prm = (ctypes.c_double * 8)(*(list(params) + [0.0] * (8 - len(params))))
    r = torch.zeros(1, dtype=torch.float64, device=image.device)
    s = _stream(stream)
    _check("binarize_bound_report", _load().binarize_bound_report(method, ptr, H, W, pitch, h, w, prm,
                                                                  r.data_ptr(), s))
    torch.cuda.synchronize(image.device)
    return float(r.item())


# ---------------------------------------------------------------- autotuner --
def autotune_window(method: int, image, h: int, w: int, k: float = 0.5, R: float = 128.0, out=None,
                    precision="fp64", W: int | None = None, stream=None):
    """Binarize (method SAUVOLA or NIBLACK) after tuning the window kernel's
    launch for this shape; returns (out, {"tile_h", "edge", "stripes", "us"})."""
    ptr, H, W, pitch = _image(image, W)
    out, op = _out(out, H, W, image.device)
    th, st_, = ctypes.c_int32(), ctypes.c_int32()
    edge, us = ctypes.c_float(), ctypes.c_float()
    _check("bz_autotune_window", _load().bz_autotune_window(
        method, ptr, H, W, pitch, h, w, k, R, out.data_ptr(), op, _PREC[precision], _stream(stream),
        ctypes.byref(th), ctypes.byref(edge), ctypes.byref(st_), ctypes.byref(us)))
    return out, {"tile_h": th.value, "edge": round(edge.value, 4), "stripes": st_.value, "us": us.value}


def autotune_quantile(image, h: int, w: int, q_num: int = 1, q_den: int = 2, offset: int = 8, out=None,
                      W: int | None = None, stream=None):
    """binarize_quantile after tuning the row-band height; returns (out, {"tile_h", "us"})."""
    ptr, H, W, pitch = _image(image, W)
    out, op = _out(out, H, W, image.device)
    th, us = ctypes.c_int32(), ctypes.c_float()
    _check("bz_autotune_quantile", _load().bz_autotune_quantile(
        ptr, H, W, pitch, h, w, q_num, q_den, offset, out.data_ptr(), op, _stream(stream),
        ctypes.byref(th), ctypes.byref(us)))
    return out, {"tile_h": th.value, "us": us.value}


def autotune_batch(jobs, precision="fp64", stream=None):
    """binarize_batch after tuning the batch tile multipliers; returns
    {"win_mult", "quant_mult", "us"}."""
    arr = (_JobC * len(jobs))(*[j.c for j in jobs])
    a, b, us = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_float()
    _check("bz_autotune_batch", _load().bz_autotune_batch(arr, len(jobs), _PREC[precision], _stream(stream),
                                                          ctypes.byref(a), ctypes.byref(b), ctypes.byref(us)))
    return {"win_mult": a.value, "quant_mult": b.value, "us": us.value}


def tune_key(gpu: str, kernel: str, cls: int, h: int, w: int, H: int, W: int) -> str:
    buf = ctypes.create_string_buffer(256)
    n = _load().bz_tune_key(gpu.encode(), kernel.encode(), cls, h, w, H, W, buf, 256)
    if n < 0:
        raise ValueError("bz_tune_key rejected its arguments")
    return buf.value.decode()


def tune_get(key: str):
    """The cached entry of `key` as a dict, or None."""
    th, st_ = ctypes.c_int32(), ctypes.c_int32()
    edge, us = ctypes.c_float(), ctypes.c_float()
    r = _load().bz_tune_get(key.encode(), ctypes.byref(th), ctypes.byref(edge), ctypes.byref(st_),
                            ctypes.byref(us))
    if r < 0:
        raise ValueError("bz_tune_get: no key")
    return None if r == 0 else {"tile_h": th.value, "edge": edge.value, "stripes": st_.value, "us": us.value}


def tune_set(key: str, tile_h: int, edge: float, stripes: int, us: float = 0.0) -> None:
    if _load().bz_tune_set(key.encode(), tile_h, edge, stripes, us) != 0:
        raise ValueError("bz_tune_set rejected the entry")


def tune_load(path: str | None = None) -> int:
    return _load().bz_tune_load(path.encode() if path else None)


def tune_save(path: str | None = None) -> int:
    return _load().bz_tune_save(path.encode() if path else None)


def tune_clear() -> None:
    _load().bz_tune_clear()


def tune_window_plan(gpu: str, precision, H: int, W: int, h: int, w: int, sms: int):
    """(cached?, {"tile_h", "edge_h", "n_edge", "tiles", "stripes", "resident"})."""
    out = (ctypes.c_int64 * 6)()
    r = _load().bz_tune_window_plan(gpu.encode(), _PREC[precision], H, W, h, w, sms, out)
    if r < 0:
        raise ValueError("bz_tune_window_plan rejected its arguments")
    names = ("tile_h", "edge_h", "n_edge", "tiles", "stripes", "resident")
    return bool(r), dict(zip(names, list(out)))

"""Python access to the CPU oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY: the plain, slow, obviously correct statement of
what the GPU library computes (Sec. 1 definitions, the Sec. 2 integral image,
the Sec. 3.1 recursive identities and Algorithm 1, the Sec. 3.4 sliding
histogram).  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package.  The GPU library never does.

Parity status: window sums, counts, FP64 thresholds, packing and quantiles are
pinned by the tests in ``tests/test_oracle_pins.py`` (three independent sum
routes, closed forms, the exact 128-bit Sauvola decision, brute-force
quantiles, hand-derived golden cases).  The FP32 threshold helper
(``threshold_f32``), which only grades the FP32 fast path by tolerance, is
pinned to the FP64 threshold within its own rounding-error bound
(``tests/test_oracle_f32_pin.py``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

SAUVOLA, NIBLACK = 0, 1
WOLF, FENG, RAIS, NICK, PHANSALKAR = 3, 4, 5, 6, 7


def build(force: bool = False) -> str:
    """Compile liboracle.so in place: C11, -O2, no FMA contraction, OpenMP."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math",
                               "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.c_void_p
    i64, i32, f64, f32 = ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_float
    sig = {
        "oracle_window_sums_bruteforce": ([P, i64, i64, i64, i32, i32, P, P, P], ctypes.c_int),
        "oracle_window_sums_integral": ([P, i64, i64, i64, i32, i32, P, P, P], ctypes.c_int),
        "oracle_window_sums_recursive": ([P, i64, i64, i64, i32, i32, P, P, P], ctypes.c_int),
        "oracle_window_sums_at": ([P, i64, i64, i64, i32, i32, P, P, i64, P, P, P], None),
        "oracle_threshold": ([i32, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32, f64, f64], f64),
        "oracle_threshold_array": ([i32, P, P, P, i64, f64, f64, P], None),
        "oracle_threshold_f32_array": ([i32, P, P, P, i64, f32, f32, P], None),
        "oracle_sauvola_bits_exact_array": ([P, P, P, P, i64, i64, i64, i64, i64, P], None),
        "oracle_sauvola_bits_paper_order_array": ([P, P, P, P, i64, f64, f64, P], None),
        "oracle_pack_bits": ([P, i64, i64, P, i64], None),
        "oracle_binarize": ([i32, P, i64, i64, i64, i32, i32, f64, f64, P, P, i64], ctypes.c_int),
        "oracle_binarize_parallel": ([i32, P, i64, i64, i64, i32, i32, f64, f64, P, i64, i32], ctypes.c_int),
        "oracle_openmp_max_threads": ([], i32),
        "oracle_window_quantile_sort": ([P, i64, i64, i64, i32, i32, i32, i32, P], ctypes.c_int),
        "oracle_window_quantile_count": ([P, i64, i64, i64, i32, i32, i32, i32, P], ctypes.c_int),
        "oracle_window_quantile_sliding": ([P, i64, i64, i64, i32, i32, i32, i32, P, i32], ctypes.c_int),
        "oracle_window_quantile_at": ([P, i64, i64, i64, i32, i32, i32, i32, P, P, i64, P], None),
        "oracle_binarize_quantile": ([P, i64, i64, i64, i32, i32, i32, i32, i32, P, P, i64, i32], ctypes.c_int),
        "oracle_window_params": ([i32, i32, P, P, P, P], None),
        "oracle_global_stats": ([P, i64, i64, i64, P, P], ctypes.c_int),
        "oracle_window_minmax_bruteforce": ([P, i64, i64, i64, i32, i32, P, P], ctypes.c_int),
        "oracle_window_minmax_deque": ([P, i64, i64, i64, i32, i32, P, P], ctypes.c_int),
        "oracle_binarize_bernsen": ([P, i64, i64, i64, i32, i32, i32, P, P, i64], ctypes.c_int),
        "oracle_window_minmax_at": ([P, i64, i64, i64, i32, i32, P, P, i64, P, P], None),
        "oracle_haar_bruteforce": ([P, i64, i64, i64, P, P, i32, P, P, i32, P], ctypes.c_int),
        "oracle_haar_integral": ([P, i64, i64, i64, P, P, i32, P, P, i32, P], ctypes.c_int),
        "oracle_threshold_ext_array": ([i32, P, P, P, i64, P, P, P], None),
        "oracle_binarize_ext": ([i32, P, i64, i64, i64, i32, i32, P, P, P, i64], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _img(img: np.ndarray, W: int | None):
    img = np.ascontiguousarray(img, dtype=np.uint8)
    H, pitch = img.shape
    W = pitch if W is None else W
    return img, H, W, pitch


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"{what}: oracle rejected its arguments (rc={rc})")


def window_params(h: int, w: int):
    """(l, r, o, u) of Algorithm 1."""
    vals = [ctypes.c_int32() for _ in range(4)]
    _load().oracle_window_params(h, w, *[ctypes.byref(v) for v in vals])
    return tuple(v.value for v in vals)


def window_sums(img: np.ndarray, h: int, w: int, route: str = "recursive", W: int | None = None):
    """(S1 uint32, S2 uint64, n uint32), each (H, W).  route: 'recursive'
    (Algorithm 1), 'bruteforce' (Sec. 1 definition) or 'integral' (Sec. 2)."""
    img, H, W, pitch = _img(img, W)
    S1 = np.empty((H, W), np.uint32)
    S2 = np.empty((H, W), np.uint64)
    n = np.empty((H, W), np.uint32)
    fn = getattr(_load(), f"oracle_window_sums_{route}")
    _check(fn(img.ctypes.data, H, W, pitch, h, w, S1.ctypes.data, S2.ctypes.data, n.ctypes.data), route)
    return S1, S2, n


def window_sums_at(img: np.ndarray, h: int, w: int, ii, jj, W: int | None = None):
    img, H, W, pitch = _img(img, W)
    ii = np.ascontiguousarray(ii, np.int64)
    jj = np.ascontiguousarray(jj, np.int64)
    if ii.size and (ii.min() < 0 or ii.max() >= H or jj.min() < 0 or jj.max() >= W):
        raise ValueError("sample position outside the image")
    S1 = np.empty(ii.size, np.uint32)
    S2 = np.empty(ii.size, np.uint64)
    n = np.empty(ii.size, np.uint32)
    _load().oracle_window_sums_at(img.ctypes.data, H, W, pitch, h, w, ii.ctypes.data, jj.ctypes.data,
                                  ii.size, S1.ctypes.data, S2.ctypes.data, n.ctypes.data)
    return S1, S2, n


def threshold(method: int, S1, S2, n, k: float, R: float = 128.0) -> np.ndarray:
    """Canonical FP64 threshold, element-wise."""
    S1 = np.ascontiguousarray(S1, np.uint32)
    S2 = np.ascontiguousarray(S2, np.uint64)
    n = np.ascontiguousarray(n, np.uint32)
    t = np.empty(S1.shape, np.float64)
    _load().oracle_threshold_array(method, S1.ctypes.data, S2.ctypes.data, n.ctypes.data, S1.size,
                                   k, R, t.ctypes.data)
    return t


def threshold_f32(method: int, S1, S2, n, k: float, R: float = 128.0) -> np.ndarray:
    """The same formula evaluated in FP32 (grades the FP32 path by tolerance;
    pinned to the FP64 threshold within its own rounding-error bound)."""
    S1 = np.ascontiguousarray(S1, np.uint32)
    S2 = np.ascontiguousarray(S2, np.uint64)
    n = np.ascontiguousarray(n, np.uint32)
    t = np.empty(S1.shape, np.float32)
    _load().oracle_threshold_f32_array(method, S1.ctypes.data, S2.ctypes.data, n.ctypes.data, S1.size,
                                       k, R, t.ctypes.data)
    return t


def sauvola_bits_exact(I, S1, S2, n, kn: int, kd: int, Rn: int, Rd: int = 1) -> np.ndarray:
    """Exact (128-bit integer) Sauvola decision for rational k and R."""
    I = np.ascontiguousarray(I, np.uint8)
    S1 = np.ascontiguousarray(S1, np.uint32)
    S2 = np.ascontiguousarray(S2, np.uint64)
    n = np.ascontiguousarray(n, np.uint32)
    bits = np.empty(S1.shape, np.uint8)
    _load().oracle_sauvola_bits_exact_array(I.ctypes.data, S1.ctypes.data, S2.ctypes.data, n.ctypes.data,
                                            S1.size, kn, kd, Rn, Rd, bits.ctypes.data)
    return bits


def sauvola_bits_paper_order(I, S1, S2, n, k: float, R: float = 128.0) -> np.ndarray:
    I = np.ascontiguousarray(I, np.uint8)
    S1 = np.ascontiguousarray(S1, np.uint32)
    S2 = np.ascontiguousarray(S2, np.uint64)
    n = np.ascontiguousarray(n, np.uint32)
    bits = np.empty(S1.shape, np.uint8)
    _load().oracle_sauvola_bits_paper_order_array(I.ctypes.data, S1.ctypes.data, S2.ctypes.data,
                                                  n.ctypes.data, S1.size, k, R, bits.ctypes.data)
    return bits


def pack_bits(bits: np.ndarray, out_pitch: int | None = None) -> np.ndarray:
    bits = np.ascontiguousarray(bits, np.uint8)
    H, W = bits.shape
    out_pitch = (W + 7) // 8 if out_pitch is None else out_pitch
    out = np.empty((H, out_pitch), np.uint8)
    _load().oracle_pack_bits(bits.ctypes.data, H, W, out.ctypes.data, out_pitch)
    return out


def binarize(method: int, img: np.ndarray, h: int, w: int, k: float, R: float = 128.0,
             W: int | None = None, out_pitch: int | None = None):
    """(bits (H, W) uint8 0/1, packed (H, out_pitch) uint8) via Algorithm 1 sums
    and the canonical FP64 threshold."""
    img, H, W, pitch = _img(img, W)
    out_pitch = (W + 7) // 8 if out_pitch is None else out_pitch
    bits = np.empty((H, W), np.uint8)
    packed = np.empty((H, out_pitch), np.uint8)
    _check(_load().oracle_binarize(method, img.ctypes.data, H, W, pitch, h, w, k, R, bits.ctypes.data,
                                   packed.ctypes.data, out_pitch), "binarize")
    return bits, packed


def sauvola(img, h, w, k=0.5, R=128.0, **kw):
    return binarize(SAUVOLA, img, h, w, k, R, **kw)


def niblack(img, h, w, k=-0.2, **kw):
    return binarize(NIBLACK, img, h, w, k, 128.0, **kw)


def binarize_parallel(method: int, img: np.ndarray, h: int, w: int, k: float, R: float = 128.0,
                      threads: int = 0, W: int | None = None) -> np.ndarray:
    """Packed output of the row-band parallel oracle (timing leg)."""
    img, H, W, pitch = _img(img, W)
    nt = threads if threads > 0 else max_threads()
    out_pitch = (W + 7) // 8
    out = np.empty((H, out_pitch), np.uint8)
    _check(_load().oracle_binarize_parallel(method, img.ctypes.data, H, W, pitch, h, w, k, R,
                                            out.ctypes.data, out_pitch, nt), "binarize_parallel")
    return out


def max_threads() -> int:
    return int(_load().oracle_openmp_max_threads())


def window_quantile(img: np.ndarray, h: int, w: int, q_num: int, q_den: int, route: str = "sliding",
                    threads: int = 1, W: int | None = None) -> np.ndarray:
    """Q (H, W) uint8.  route: 'sort' or 'count' (brute force) or 'sliding'."""
    img, H, W, pitch = _img(img, W)
    Q = np.empty((H, W), np.uint8)
    lib = _load()
    if route == "sliding":
        rc = lib.oracle_window_quantile_sliding(img.ctypes.data, H, W, pitch, h, w, q_num, q_den,
                                                Q.ctypes.data, threads)
    else:
        rc = getattr(lib, f"oracle_window_quantile_{route}")(img.ctypes.data, H, W, pitch, h, w,
                                                             q_num, q_den, Q.ctypes.data)
    _check(rc, "window_quantile")
    return Q


def window_quantile_at(img: np.ndarray, h: int, w: int, q_num: int, q_den: int, ii, jj,
                       W: int | None = None) -> np.ndarray:
    img, H, W, pitch = _img(img, W)
    ii = np.ascontiguousarray(ii, np.int64)
    jj = np.ascontiguousarray(jj, np.int64)
    if ii.size and (ii.min() < 0 or ii.max() >= H or jj.min() < 0 or jj.max() >= W):
        raise ValueError("sample position outside the image")
    Q = np.empty(ii.size, np.uint8)
    _load().oracle_window_quantile_at(img.ctypes.data, H, W, pitch, h, w, q_num, q_den,
                                      ii.ctypes.data, jj.ctypes.data, ii.size, Q.ctypes.data)
    return Q


def binarize_quantile(img: np.ndarray, h: int, w: int, q_num: int, q_den: int, offset: int = 8,
                      threads: int = 1, W: int | None = None, out_pitch: int | None = None):
    img, H, W, pitch = _img(img, W)
    out_pitch = (W + 7) // 8 if out_pitch is None else out_pitch
    bits = np.empty((H, W), np.uint8)
    packed = np.empty((H, out_pitch), np.uint8)
    _check(_load().oracle_binarize_quantile(img.ctypes.data, H, W, pitch, h, w, q_num, q_den, offset,
                                            bits.ctypes.data, packed.ctypes.data, out_pitch, threads),
           "binarize_quantile")
    return bits, packed


# ---------------------------------------------------------------- Table 1 --
def params(k: float = 0.5, R: float = 128.0, alpha1: float = 0.88, k1: float = 0.25,
           k2: float = 0.04, gamma: float = 2.0, p: float = 2.0, q: float = 10.0 / 255.0) -> np.ndarray:
    """The parameter vector of the Table 1 thresholds: {k, R, alpha1, k1, k2, gamma, p, q}."""
    return np.array([k, R, alpha1, k1, k2, gamma, p, q], np.float64)


def global_stats(img: np.ndarray, W: int | None = None):
    """((L, M, S) as float64, (sum, sumsq, N) as ints): Table 1's global
    minimum, mean and population standard deviation."""
    img, H, W, pitch = _img(img, W)
    st = np.empty(3, np.float64)
    sums = np.empty(3, np.uint64)
    _check(_load().oracle_global_stats(img.ctypes.data, H, W, pitch, st.ctypes.data, sums.ctypes.data),
           "global_stats")
    return st, tuple(int(v) for v in sums)


def threshold_ext(method: int, S1, S2, n, prm, glob) -> np.ndarray:
    """Canonical FP64 threshold of any Table 1 method, element-wise; glob = (L, M, S)."""
    S1 = np.ascontiguousarray(S1, np.uint32)
    S2 = np.ascontiguousarray(S2, np.uint64)
    n = np.ascontiguousarray(n, np.uint32)
    prm = np.ascontiguousarray(prm, np.float64)
    glob = np.ascontiguousarray(glob, np.float64)
    t = np.empty(S1.shape, np.float64)
    _load().oracle_threshold_ext_array(method, S1.ctypes.data, S2.ctypes.data, n.ctypes.data, S1.size,
                                       prm.ctypes.data, glob.ctypes.data, t.ctypes.data)
    return t


def binarize_ext(method: int, img: np.ndarray, h: int, w: int, prm, W: int | None = None,
                 out_pitch: int | None = None):
    """(bits, packed) of any Table 1 method (global statistics + Algorithm 1
    sums + canonical FP64 threshold)."""
    img, H, W, pitch = _img(img, W)
    out_pitch = (W + 7) // 8 if out_pitch is None else out_pitch
    prm = np.ascontiguousarray(prm, np.float64)
    bits = np.empty((H, W), np.uint8)
    packed = np.empty((H, out_pitch), np.uint8)
    _check(_load().oracle_binarize_ext(method, img.ctypes.data, H, W, pitch, h, w, prm.ctypes.data,
                                       bits.ctypes.data, packed.ctypes.data, out_pitch), "binarize_ext")
    return bits, packed


# ------------------------------------------------------- local min / max --
def window_minmax(img: np.ndarray, h: int, w: int, route: str = "deque", W: int | None = None):
    """(min, max) of the clipped window, each (H, W) uint8.  route: 'deque'
    (separable monotonic deques) or 'bruteforce' (direct loops)."""
    img, H, W, pitch = _img(img, W)
    mn = np.empty((H, W), np.uint8)
    mx = np.empty((H, W), np.uint8)
    fn = getattr(_load(), f"oracle_window_minmax_{route}")
    _check(fn(img.ctypes.data, H, W, pitch, h, w, mn.ctypes.data, mx.ctypes.data), route)
    return mn, mx


def window_minmax_at(img: np.ndarray, h: int, w: int, ii, jj, W: int | None = None):
    img, H, W, pitch = _img(img, W)
    ii = np.ascontiguousarray(ii, np.int64)
    jj = np.ascontiguousarray(jj, np.int64)
    if ii.size and (ii.min() < 0 or ii.max() >= H or jj.min() < 0 or jj.max() >= W):
        raise ValueError("sample position outside the image")
    mn = np.empty(ii.size, np.uint8)
    mx = np.empty(ii.size, np.uint8)
    _load().oracle_window_minmax_at(img.ctypes.data, H, W, pitch, h, w, ii.ctypes.data, jj.ctypes.data,
                                    ii.size, mn.ctypes.data, mx.ctypes.data)
    return mn, mx


def binarize_bernsen(img: np.ndarray, h: int, w: int, contrast_limit: int = 15, W: int | None = None,
                     out_pitch: int | None = None):
    """(bits, packed) of Bernsen's midrange threshold with a contrast limit."""
    img, H, W, pitch = _img(img, W)
    out_pitch = (W + 7) // 8 if out_pitch is None else out_pitch
    bits = np.empty((H, W), np.uint8)
    packed = np.empty((H, out_pitch), np.uint8)
    _check(_load().oracle_binarize_bernsen(img.ctypes.data, H, W, pitch, h, w, contrast_limit,
                                           bits.ctypes.data, packed.ctypes.data, out_pitch),
           "binarize_bernsen")
    return bits, packed


# --------------------------------------------------------- Haar-like sums --
def haar(img: np.ndarray, rows, cols, route: str = "integral", W: int | None = None) -> np.ndarray:
    """Separable piecewise-constant window sum, int32 (H, W).  rows / cols:
    lists of (length, weight) segments of the window's rows / columns
    (h = sum of row lengths, w = sum of column lengths, placed as in
    Algorithm 1).  route: 'integral' (four lookups per rectangle) or
    'bruteforce' (direct loops)."""
    img, H, W, pitch = _img(img, W)
    rl = np.ascontiguousarray([r[0] for r in rows], np.int32)
    rw = np.ascontiguousarray([r[1] for r in rows], np.int32)
    cl = np.ascontiguousarray([c[0] for c in cols], np.int32)
    cw = np.ascontiguousarray([c[1] for c in cols], np.int32)
    out = np.empty((H, W), np.int32)
    fn = getattr(_load(), f"oracle_haar_{route}")
    _check(fn(img.ctypes.data, H, W, pitch, rl.ctypes.data, rw.ctypes.data, len(rows), cl.ctypes.data,
              cw.ctypes.data, len(cols), out.ctypes.data), "haar")
    return out

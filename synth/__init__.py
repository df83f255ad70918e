"""Seeded synthetic document images (inputs for both the GPU library and the
oracle).  Holds no binarization arithmetic.

The C source ``docgen.c`` is compiled in place on first use (or by
``build()``), so the same bytes come out on x86-64 and aarch64 hosts.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "docgen.c")
_LIB = os.path.join(_HERE, "libdocgen.so")
_lib = None

# Seeds of the standard workloads: workload c uses BASE_SEED + c and image b
# of a batch uses that seed + b.
BASE_SEED = 0x19051303800


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i64, u64, i32, f64 = ctypes.c_int64, ctypes.c_uint64, ctypes.c_int32, ctypes.c_double
        lib.synth_document.argtypes = [ctypes.c_void_p, i64, i64, i64, u64, i32, f64, f64, f64]
        lib.synth_document.restype = ctypes.c_int
        lib.synth_uniform.argtypes = [ctypes.c_void_p, i64, i64, i64, u64, i32, i32]
        lib.synth_uniform.restype = ctypes.c_int
        lib.synth_splitmix64.argtypes = [u64, ctypes.c_void_p, i64]
        lib.synth_splitmix64.restype = None
        _lib = lib
    return _lib


def document(H: int, W: int, seed: int, *, stains: int = 0, stroke_frac: float = 0.10,
             sigma: float = 8.0, salt_pepper: float = 0.0, pitch: int | None = None) -> np.ndarray:
    """uint8 array of shape (H, pitch) whose first W columns hold the image."""
    pitch = W if pitch is None else pitch
    out = np.empty((H, pitch), dtype=np.uint8)
    rc = _load().synth_document(out.ctypes.data, H, W, pitch, seed & (2**64 - 1), stains,
                                stroke_frac, sigma, salt_pepper)
    if rc != 0:
        raise ValueError(f"synth_document rejected H={H} W={W} pitch={pitch} (rc={rc})")
    return out


def uniform(H: int, W: int, seed: int, lo: int = 0, hi: int = 255, pitch: int | None = None) -> np.ndarray:
    pitch = W if pitch is None else pitch
    out = np.empty((H, pitch), dtype=np.uint8)
    rc = _load().synth_uniform(out.ctypes.data, H, W, pitch, seed & (2**64 - 1), lo, hi)
    if rc != 0:
        raise ValueError("synth_uniform rejected its arguments")
    return out


def splitmix64(seed: int, count: int) -> np.ndarray:
    out = np.empty(count, dtype=np.uint64)
    _load().synth_splitmix64(seed & (2**64 - 1), out.ctypes.data, count)
    return out


# ---- the standard workloads ---------------------------------------------------------
def single_page(seed_offset: int = 0) -> np.ndarray:
    """512 x 384 page (W=512, H=384): gradient, strokes, noise."""
    return document(384, 512, BASE_SEED + 0 + seed_offset)


def large_page(seed_offset: int = 0) -> np.ndarray:
    """4096 x 3072 page (12,582,912 px) with three stains."""
    return document(3072, 4096, BASE_SEED + 1 + seed_offset, stains=3)


def quantile_page(seed_offset: int = 0) -> np.ndarray:
    """2048 x 2048 page with three stains and 2% salt-and-pepper noise."""
    return document(2048, 2048, BASE_SEED + 2 + seed_offset, stains=3, salt_pepper=0.02)


BATCH_WINDOWS = (15, 31, 63, 127)


def batch_specs(count: int = 256, seed: int = BASE_SEED + 3):
    """Shapes, windows and methods of the uneven batch: sizes log-uniform on the
    diagonal between 320x240 and 2480x3508, window h=w from {15,31,63,127},
    method Sauvola (0) or Niblack (1).  Returns a list of dicts."""
    z = splitmix64(seed, 3 * count)
    specs = []
    for b in range(count):
        uu = float(z[3 * b] >> np.uint64(11)) / 2.0**53
        W = int(round(320 * (2480 / 320) ** uu))
        H = int(round(240 * (3508 / 240) ** uu))
        win = BATCH_WINDOWS[int(z[3 * b + 1] % np.uint64(4))]
        method = int(z[3 * b + 2] % np.uint64(2))
        specs.append({"H": H, "W": W, "h": win, "w": win, "method": method, "seed": seed + 1000 + b})
    return specs

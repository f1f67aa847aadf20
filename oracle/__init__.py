"""FP64 CPU oracle of the spectral DPSR layer (Shape As Points, Sec. 3.1 and
supplementary Sec. A). TEST INFRASTRUCTURE: only the tests, the smoke check and
the CPU-baseline leg of the benchmark load it.

The arithmetic lives in ``dpsr_oracle.c`` (plain C, its own radix-2 FFT). This
module compiles it with gcc on first use and wraps it with ctypes over float64
numpy arrays. It imports nothing from the GPU package.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dpsr_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

ORACLE_OK = 0
ORACLE_EINVAL = -1
ORACLE_ENOMEM = -2
ORACLE_EDEGENERATE = -4


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what} failed with oracle status {code}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile dpsr_oracle.c into oracle/_build/liboracle.so (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # ORACLE_LIB points the tests that plant mistakes at a mutated copy.
            lib = ctypes.CDLL(os.environ.get("ORACLE_LIB") or build())
            dp = ctypes.POINTER(ctypes.c_double)
            i64 = ctypes.c_int64
            lib.oracle_fft3.argtypes = [ctypes.c_int, dp, ctypes.c_int]
            lib.oracle_splat.argtypes = [ctypes.c_int, i64, dp, dp, ctypes.c_int, dp]
            lib.oracle_gather.argtypes = [ctypes.c_int, i64, dp, dp, dp]
            lib.oracle_dpsr_forward.argtypes = [ctypes.c_int, ctypes.c_double, i64, dp, dp,
                                                dp, dp, dp]
            lib.oracle_dpsr_backward.argtypes = [ctypes.c_int, ctypes.c_double, i64, dp, dp,
                                                 dp, dp, dp]
            lib.oracle_dpsr_backward_terms.argtypes = [ctypes.c_int, ctypes.c_double, i64, dp, dp,
                                                       dp, dp, dp, dp]
            lib.oracle_dpsr_forward_box.argtypes = [ctypes.c_int, ctypes.c_double, i64, dp, dp, dp,
                                                    dp, dp, dp]
            lib.oracle_dpsr_backward_box.argtypes = [ctypes.c_int, ctypes.c_double, i64, dp, dp, dp,
                                                     dp, dp, dp]
            for f in ("oracle_dpsr_forward_box", "oracle_dpsr_backward_box", "oracle_dpsr_backward_terms", "oracle_fft3", "oracle_splat", "oracle_gather", "oracle_dpsr_forward",
                      "oracle_dpsr_backward", "oracle_threads", "oracle_set_threads"):
                getattr(lib, f).restype = ctypes.c_int
            lib.oracle_threads.argtypes = []
            lib.oracle_set_threads.argtypes = [ctypes.c_int]
            lib.oracle_set_threads.restype = None
            _lib = lib
    return _lib


def _p(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def _check(code, what):
    if code != ORACLE_OK:
        raise OracleError(code, what)


def threads() -> int:
    """OpenMP threads the oracle uses (its FFT pencils run in parallel)."""
    return int(_load().oracle_threads())


def set_threads(n: int) -> None:
    """Threads for the oracle's parallel loops from now on."""
    _load().oracle_set_threads(int(n))


def fft3(g: np.ndarray, inverse: bool = False) -> np.ndarray:
    """3D DFT of a complex r^3 grid: forward unnormalised (Eq. A3), inverse
    with 1/r^3 (Eq. A4)."""
    r = g.shape[0]
    a = np.ascontiguousarray(np.asarray(g, dtype=np.complex128)).copy()
    buf = a.view(np.float64)
    _check(_load().oracle_fft3(r, _p(buf), 1 if inverse else 0), "oracle_fft3")
    return a


def splat(r: int, points, values=None) -> np.ndarray:
    """Inverse trilinear splat (Eq. A2). values: N x C, or None for the weight
    field W (splat of ones). Returns C x r^3 (or r^3 for C = 1 / None)."""
    pts = _f64(points, (-1, 3))
    if values is None:
        nch, vals = 1, None
    else:
        vals = _f64(values)
        vals = vals.reshape(pts.shape[0], -1)
        nch = vals.shape[1]
    out = np.zeros((nch, r, r, r), np.float64)
    _check(_load().oracle_splat(r, pts.shape[0], _p(pts), _p(vals), nch, _p(out)), "oracle_splat")
    return out[0] if nch == 1 else out


def gather(grid, points) -> np.ndarray:
    """Trilinear lookup of a real r^3 grid at the points."""
    g = _f64(grid)
    pts = _f64(points, (-1, 3))
    out = np.zeros(pts.shape[0], np.float64)
    _check(_load().oracle_gather(g.shape[0], pts.shape[0], _p(pts), _p(g), _p(out)),
           "oracle_gather")
    return out


def forward(r: int, sigma: float, points, normals, full: bool = False, box=None):
    """DPSR forward (Eq. 3, Eq. 4). Returns chi (r^3), or with full=True the
    tuple (chi, chi_prime, mu, s). box: side lengths (L0, L1, L2) of the
    periodic domain (default the unit cube); points in box coordinates."""
    pts = _f64(points, (-1, 3))
    nrm = _f64(normals, (-1, 3))
    chi = np.zeros((r, r, r), np.float64)
    chip = np.zeros((r, r, r), np.float64) if full else None
    mus = np.zeros(2, np.float64)
    if box is None:
        _check(_load().oracle_dpsr_forward(r, float(sigma), pts.shape[0], _p(pts), _p(nrm), _p(chi),
                                           _p(chip), _p(mus)), "oracle_dpsr_forward")
    else:
        b = _f64(box, (3,))
        _check(_load().oracle_dpsr_forward_box(r, float(sigma), pts.shape[0], _p(pts), _p(nrm), _p(b),
                                               _p(chi), _p(chip), _p(mus)), "oracle_dpsr_forward_box")
    if full:
        return chi, chip, float(mus[0]), float(mus[1])
    return chi


def backward(r: int, sigma: float, points, normals, dchi, mean_term: bool = False, box=None):
    """DPSR backward: (dL/dpoints, dL/dnormals), each N x 3. With
    mean_term=True also the part of dL/dpoints that flows through the mean of
    Eq. 4, as a third array. box: as for forward (not with mean_term)."""
    pts = _f64(points, (-1, 3))
    nrm = _f64(normals, (-1, 3))
    g = _f64(dchi, (r, r, r))
    dp = np.zeros_like(pts)
    dn = np.zeros_like(nrm)
    if box is not None:
        if mean_term:
            raise ValueError("mean_term is for the unit cube")
        b = _f64(box, (3,))
        _check(_load().oracle_dpsr_backward_box(r, float(sigma), pts.shape[0], _p(pts), _p(nrm), _p(b),
                                                _p(g), _p(dp), _p(dn)), "oracle_dpsr_backward_box")
        return dp, dn
    if mean_term:
        dm = np.zeros_like(pts)
        _check(_load().oracle_dpsr_backward_terms(r, float(sigma), pts.shape[0], _p(pts), _p(nrm),
                                                  _p(g), _p(dp), _p(dn), _p(dm)),
               "oracle_dpsr_backward_terms")
        return dp, dn, dm
    _check(_load().oracle_dpsr_backward(r, float(sigma), pts.shape[0], _p(pts), _p(nrm), _p(g),
                                        _p(dp), _p(dn)), "oracle_dpsr_backward")
    return dp, dn

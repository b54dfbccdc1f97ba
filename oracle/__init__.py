"""FP64 CPU oracle for the lensed-image simulation path (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` are the only callers.  The product library never loads this
module and shares no code with it.  The arithmetic lives in ``lens_oracle.cpp``;
this wrapper only marshals NumPy arrays and the plain system description drawn by
the shared input generators.

Functions whose result is pinned by the physics tests (``tests/test_oracle_pins.py``):
every deflection profile, the Sersic source, the grid and bin-down, the PSF
convolution and its transpose, and the likelihood gradient.  Nothing here is
"parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lens_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liblensoracle.so")

LENS_CODES = {"SIS": 0, "SIE": 1, "EPL": 2, "SHEAR": 3, "POINT_MASS": 4, "NFW": 5, "TNFW": 6,
              "EPL_E1E2": 7, "SIE_E1E2": 8, "MULTIPOLE": 9, "EPL_MULTIPOLE_M1M3M4": 10, "CSE": 11,
              "NFW_ELLIPSE_CSE": 12, "HERNQUIST_ELLIPSE_CSE": 13, "MULTIPOLE_ELL": 14}
LIGHT_CODES = {"SERSIC_ELLIPSE_Q_PHI": 0, "SERSIC_ELLIPSE": 1, "SERSIC": 2, "SHAPELETS": 3}
DEFL_PARAMS = 12   # parameters per deflector in the oracle's layout

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (FP64, IEEE, OpenMP) into oracle/_build."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


class _OSys(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("s", ctypes.c_int),
                ("dpix", ctypes.c_double), ("x0", ctypes.c_double), ("y0", ctypes.c_double),
                ("n_defl", ctypes.c_int),
                ("defl_type", ctypes.POINTER(ctypes.c_int)),
                ("defl_p", ctypes.POINTER(ctypes.c_double)),
                ("n_sub", ctypes.c_int),
                ("sub", ctypes.POINTER(ctypes.c_double)),
                ("src_type", ctypes.c_int),
                ("src_p", ctypes.c_double * 8),
                ("k", ctypes.c_int),
                ("psf", ctypes.POINTER(ctypes.c_double)),
                ("src_coef", ctypes.POINTER(ctypes.c_double)),
                ("n_src_coef", ctypes.c_int)]


_dp = ctypes.POINTER(ctypes.c_double)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.oracle_alpha.argtypes = [ctypes.c_int, _dp, ctypes.c_int, _dp, _dp, _dp, _dp]
            L.oracle_light.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]
            L.oracle_alpha_system.argtypes = [ctypes.POINTER(_OSys), ctypes.c_int, _dp, _dp, _dp, _dp,
                                              ctypes.c_int]
            L.oracle_image_rows.argtypes = [ctypes.POINTER(_OSys), ctypes.c_int, ctypes.c_int, _dp,
                                            ctypes.c_int]
            L.oracle_image.argtypes = [ctypes.POINTER(_OSys), _dp, _dp, ctypes.c_int]
            L.oracle_convolve.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int, _dp]
            L.oracle_correlate.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int, _dp]
            L.oracle_loglike.argtypes = [ctypes.POINTER(_OSys), _dp, ctypes.c_double, ctypes.c_double,
                                         _dp, ctypes.c_int, _dp, _dp, ctypes.c_int]
            L.oracle_model_image.argtypes = [ctypes.POINTER(_OSys), _dp, _dp]
            L.oracle_set_threads.argtypes = [ctypes.c_int]
            L.oracle_nthreads.restype = ctypes.c_int
            _lib = L
    return _lib


def _ptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    return a.ctypes.data_as(_dp)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def set_threads(n: int) -> None:
    lib().oracle_set_threads(int(n))


def nthreads() -> int:
    return int(lib().oracle_nthreads())


class _Packed:
    """Keeps the FP64 copies alive while the C struct points at them."""

    def __init__(self, system):
        g = system.grid
        self.types = np.array([LENS_CODES[n] for n, _ in system.deflectors] or [0], np.int32)
        p = np.zeros((max(len(system.deflectors), 1), DEFL_PARAMS))
        for i, (_, vals) in enumerate(system.deflectors):
            p[i, :len(vals)] = vals
        self.p = np.ascontiguousarray(p)
        self.sub = _f64(system.subhalos).reshape(5, -1).copy()
        self.psf = _f64(system.psf) if system.psf is not None else np.zeros(1)
        k = 0 if system.psf is None else int(system.psf.shape[0])
        st = _OSys()
        st.nx, st.ny, st.s = g.nx, g.ny, g.s
        st.dpix, st.x0, st.y0 = float(g.dpix), float(g.x0), float(g.y0)
        st.n_defl = len(system.deflectors)
        st.defl_type = self.types.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        st.defl_p = _ptr(self.p)
        st.n_sub = int(self.sub.shape[1])
        st.sub = _ptr(self.sub)
        st.src_type = LIGHT_CODES[system.source[0]]
        for i, v in enumerate(system.source[1]):
            st.src_p[i] = float(v)
        st.k = k
        st.psf = _ptr(self.psf)
        coef = getattr(system, "source_coeffs", None)
        self.coef = _f64(coef).ravel().copy() if coef is not None else np.zeros(1)
        st.src_coef = _ptr(self.coef)
        st.n_src_coef = 0 if coef is None else int(self.coef.size)
        self.st = st


def alpha(name: str, params, x, y) -> Tuple[np.ndarray, np.ndarray]:
    """Deflection of one profile at points (x, y)."""
    p = np.zeros(DEFL_PARAMS)
    p[:len(params)] = params
    x = _f64(x).ravel(); y = _f64(y).ravel()
    ax = np.empty_like(x); ay = np.empty_like(x)
    rc = lib().oracle_alpha(LENS_CODES[name], _ptr(p), x.size, _ptr(x), _ptr(y), _ptr(ax), _ptr(ay))
    if rc != 0:
        raise ValueError(f"oracle_alpha failed for {name}")
    return ax, ay


def light(name: str, params, x, y, coeffs=None) -> np.ndarray:
    """Source surface brightness of one light profile at points (x, y) (SHAPELETS: with its
    amplitudes `coeffs`)."""
    p = np.zeros(8)
    p[:len(params)] = params
    x = _f64(x).ravel(); y = _f64(y).ravel()
    out = np.empty_like(x)
    c = _f64(coeffs).ravel().copy() if coeffs is not None else np.zeros(1)
    nc = 0 if coeffs is None else int(c.size)
    if lib().oracle_light(LIGHT_CODES[name], _ptr(p), _ptr(c), nc, x.size, _ptr(x), _ptr(y), _ptr(out)) != 0:
        raise ValueError(f"oracle_light failed for {name}")
    return out


def alpha_system(system, x, y, fp32: bool = False) -> Tuple[np.ndarray, np.ndarray]:
    """Total deflection (deflector list + all subhalos) at points (x, y)."""
    pk = _Packed(system)
    x = _f64(x).ravel(); y = _f64(y).ravel()
    ax = np.empty_like(x); ay = np.empty_like(x)
    if lib().oracle_alpha_system(ctypes.byref(pk.st), x.size, _ptr(x), _ptr(y), _ptr(ax), _ptr(ay),
                                 int(fp32)) != 0:
        raise ValueError("oracle_alpha_system failed")
    return ax, ay


def image_rows(system, row0: int, row1: int, fp32: bool = False) -> np.ndarray:
    """Unconvolved (binned) image rows [row0, row1)."""
    pk = _Packed(system)
    out = np.empty((row1 - row0, system.grid.nx))
    if lib().oracle_image_rows(ctypes.byref(pk.st), row0, row1, _ptr(out), int(fp32)) != 0:
        raise ValueError("oracle_image_rows failed")
    return out


def image(system, fp32: bool = False, return_unconvolved: bool = False):
    """Full simulated image (PSF-convolved if the system has a PSF)."""
    pk = _Packed(system)
    g = system.grid
    out = np.empty((g.ny, g.nx))
    raw = np.empty((g.ny, g.nx))
    if lib().oracle_image(ctypes.byref(pk.st), _ptr(out), _ptr(raw), int(fp32)) != 0:
        raise ValueError("oracle_image failed")
    return (out, raw) if return_unconvolved else out


def convolve(img, K) -> np.ndarray:
    img = _f64(img); K = _f64(K)
    out = np.empty_like(img)
    if lib().oracle_convolve(_ptr(img), img.shape[0], img.shape[1], _ptr(K), K.shape[0], _ptr(out)) != 0:
        raise ValueError("bad kernel")
    return out


def correlate(img, K) -> np.ndarray:
    img = _f64(img); K = _f64(K)
    out = np.empty_like(img)
    if lib().oracle_correlate(_ptr(img), img.shape[0], img.shape[1], _ptr(K), K.shape[0], _ptr(out)) != 0:
        raise ValueError("bad kernel")
    return out


def loglike(system, data, sigma_bkg: float, t_exp: float, params, grad: bool = True, fp32: bool = False):
    """Chi^2 log-likelihood (and its exact gradient) at [n, 15] parameter points.

    fp32=True is the conditioning-floor mode: grid, deflection terms, traced positions and
    model image rounded to FP32 (values only), the error any FP32 evaluation must make."""
    pk = _Packed(system)
    P = _f64(params).reshape(-1, 15)
    d = _f64(data)
    n = P.shape[0]
    L = np.empty(n)
    G = np.empty((n, 15)) if grad else None
    if lib().oracle_loglike(ctypes.byref(pk.st), _ptr(d), float(sigma_bkg), float(t_exp), _ptr(P), n,
                            _ptr(L), _ptr(G), int(fp32)) != 0:
        raise ValueError("oracle_loglike failed")
    return (L, G) if grad else L


def model_image(system, params) -> np.ndarray:
    """PSF-convolved model image at one 15-parameter point (fixed subhalos)."""
    pk = _Packed(system)
    P = _f64(params).ravel()
    g = system.grid
    out = np.empty((g.ny, g.nx))
    if lib().oracle_model_image(ctypes.byref(pk.st), _ptr(P), _ptr(out)) != 0:
        raise ValueError("oracle_model_image failed")
    return out


def linear_amp(system, data, sigma_bkg: float, t_exp: float, params):
    """Weighted least-squares source amplitude per parameter point: with w = 1/(sigma_bkg^2 +
    max(d, 0)/t_exp) and m1 the model at unit amplitude, amp = sum w d m1 / sum w m1^2, and the
    log-likelihood at it, -1/2 sum w (d - amp m1)^2 (straight from the definitions, FP64)."""
    P = _f64(params).reshape(-1, 15)
    d = _f64(data)
    w = 1.0 / (sigma_bkg ** 2 + np.maximum(d, 0.0) / t_exp)
    amps, logLs = [], []
    for p in P:
        q = p.copy()
        q[8] = 1.0
        m1 = model_image(system, q)
        a = np.sum(w * d * m1) / np.sum(w * m1 * m1)
        amps.append(a)
        logLs.append(-0.5 * np.sum(w * (d - a * m1) ** 2))
    return np.array(amps), np.array(logLs)

"""Thin ctypes binding of liblenssim.so (include/lens_sim.h).

Argument marshalling only: every step of the simulation runs in the CUDA library.
PyTorch supplies device memory and the current CUDA stream.  If the library has not
been built, every entry point raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np
import torch

from . import workloads as W

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "liblenssim.so")

LENS_OK, LENS_ERR_INVALID_ARG, LENS_ERR_OOM, LENS_ERR_CUDA = 0, -1, -2, -3
LENS_ERR_TIMEOUT, LENS_ERR_BUSY, LENS_ERR_UNSUPPORTED, LENS_ERR_CANCELLED = -4, -5, -6, -7
STATUS_NAMES = {0: "LENS_OK", -1: "LENS_ERR_INVALID_ARG", -2: "LENS_ERR_OOM", -3: "LENS_ERR_CUDA",
                -4: "LENS_ERR_TIMEOUT", -5: "LENS_ERR_BUSY", -6: "LENS_ERR_UNSUPPORTED",
                -7: "LENS_ERR_CANCELLED"}

LENS_TYPES = {"SIS": 0, "SIE": 1, "EPL": 2, "SHEAR": 3, "POINT_MASS": 4, "NFW": 5, "TNFW": 6,
              "EPL_E1E2": 7, "SIE_E1E2": 8, "MULTIPOLE": 9, "EPL_MULTIPOLE_M1M3M4": 10, "CSE": 11,
              "NFW_ELLIPSE_CSE": 12, "HERNQUIST_ELLIPSE_CSE": 13, "MULTIPOLE_ELL": 14}
LIGHT_TYPES = {"SERSIC_ELLIPSE_Q_PHI": 0, "SERSIC_ELLIPSE": 1, "SERSIC": 2, "SHAPELETS": 3}
MAX_DEFLECTORS = 8
CONV_METHODS = {"auto": 0, "direct": 1, "fft": 2}
CONV_FFT_MIN_K = 33   # LENS_CONV_FFT_MIN_K: auto takes the FFT from this kernel size on
TRACE_VARIANTS = ("cta8", "cta4x2pass", "cluster2x4", "cluster4x2", "cluster8x1")
BATCH_FORMS = ("cta4x2pass", "cta8", "cluster2x4")   # LENS_BATCH_FORMS persistent trace kernels
BATCH_ORDERS = ("cost_desc", "given")
# LENS_PIPE_RATES entries of lens_sim_pipe_rates, in order (per SM and SM clock)
PIPE_RATES = ("fp32_lane_ops_ffma2", "fp32_lane_ops_ffma", "mufu_rsqrt", "mufu_ex2", "mufu_lg2", "mufu_rcp")
_TUNE_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")

EXPORTED = ("lens_sim_create", "lens_sim_destroy", "lens_sim_last_error", "lens_sim_register_psf",
            "lens_sim_register_subhalos", "lens_sim_image", "lens_sim_deflection", "lens_sim_convolve",
            "lens_sim_autotune", "lens_sim_set_variant", "lens_sim_set_far_field", "lens_sim_set_batch_schedule",
            "lens_sim_autotune_batch",
            "lens_sim_set_conv_method", "lens_sim_grad",
            "lens_sim_linear_amp", "lens_sim_pipe_rates",
            "lens_sim_image_noalloc", "lens_serve_create", "lens_serve_sim", "lens_serve_submit", "lens_serve_wait",
            "lens_serve_poll", "lens_serve_cancel", "lens_serve_pause", "lens_serve_stats", "lens_serve_last_error",
            "lens_serve_reset_stats", "lens_serve_destroy")


PROFILE_PARAMS = 12   # floats in lens_profile.p


class LensProfile(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("p", ctypes.c_float * PROFILE_PARAMS)]


class LightProfile(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("p", ctypes.c_float * 8)]


class LensGrid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("supersample", ctypes.c_int),
                ("pixel_scale", ctypes.c_float), ("x0", ctypes.c_float), ("y0", ctypes.c_float)]


class LensSystemC(ctypes.Structure):
    _fields_ = [("grid", LensGrid),
                ("deflectors", ctypes.POINTER(LensProfile)),
                ("n_deflectors", ctypes.c_int),
                ("subhalos", ctypes.c_void_p),
                ("n_subhalos", ctypes.c_int),
                ("subhalo_table", ctypes.c_int),
                ("source", LightProfile),
                ("psf_id", ctypes.c_int),
                ("source_coeffs", ctypes.POINTER(ctypes.c_float)),
                ("n_source_coeffs", ctypes.c_int)]


class SimConfig(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("mem_budget_bytes", ctypes.c_size_t),
                ("max_batch", ctypes.c_int), ("flags", ctypes.c_uint)]


class LensRequest(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("sys", LensSystemC), ("data", ctypes.c_void_p),
                ("sigma_bkg", ctypes.c_float), ("t_exp", ctypes.c_float), ("params", ctypes.c_void_p),
                ("out", ctypes.c_void_p), ("out_grad", ctypes.c_void_p)]


class LensSimError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _LIB_PATH


def lib():
    """Load liblenssim.so; raise if it has not been built (no fallback path exists)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIB_PATH):
                raise RuntimeError(f"CUDA library {_LIB_PATH} is missing: run "
                                   "`python -c 'import __graft_entry__ as g; g.build()'` first")
            L = ctypes.CDLL(_LIB_PATH)
            vp, ip, fp = ctypes.c_void_p, ctypes.c_int, ctypes.c_float
            L.lens_sim_create.argtypes = [ctypes.POINTER(SimConfig), ctypes.POINTER(vp)]
            L.lens_sim_destroy.argtypes = [vp]
            L.lens_sim_destroy.restype = None
            L.lens_sim_last_error.argtypes = [vp]
            L.lens_sim_last_error.restype = ctypes.c_char_p
            L.lens_sim_register_psf.argtypes = [vp, vp, ip, ctypes.POINTER(ip)]
            L.lens_sim_register_subhalos.argtypes = [vp, vp, ip, ctypes.POINTER(ip)]
            L.lens_sim_image.argtypes = [vp, ctypes.POINTER(LensSystemC), ip, ctypes.POINTER(vp), vp]
            L.lens_sim_deflection.argtypes = [vp, ctypes.POINTER(LensSystemC), vp, vp, ip, vp, vp, vp]
            L.lens_sim_convolve.argtypes = [vp, vp, ip, ip, ip, ip, vp, vp]
            L.lens_sim_grad.argtypes = [vp, ctypes.POINTER(LensSystemC), vp, fp, fp, vp, ip, vp, vp, vp]
            L.lens_sim_autotune.argtypes = [vp, ctypes.POINTER(LensSystemC), ip, ctypes.POINTER(ip),
                                            ctypes.POINTER(fp), ip, vp]
            L.lens_sim_set_variant.argtypes = [vp, ip]
            L.lens_sim_set_far_field.argtypes = [vp, ctypes.c_float]
            L.lens_sim_set_batch_schedule.argtypes = [vp, ip, ip]
            L.lens_sim_autotune_batch.argtypes = [vp, ctypes.POINTER(LensSystemC), ip, ctypes.POINTER(vp), ip,
                                                  ctypes.POINTER(ip), ctypes.POINTER(ip), ctypes.POINTER(fp), vp]
            L.lens_sim_set_conv_method.argtypes = [vp, ctypes.c_int]
            L.lens_sim_pipe_rates.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ip]
            L.lens_sim_image_noalloc.argtypes = [ctypes.POINTER(LensSystemC), vp, ip, vp, vp]
            L.lens_sim_linear_amp.argtypes = [vp, ctypes.POINTER(LensSystemC), vp, fp, fp, vp, ip, vp, vp, vp]
            L.lens_serve_create.argtypes = [ctypes.POINTER(SimConfig), ip, ctypes.POINTER(vp)]
            L.lens_serve_sim.argtypes = [vp]
            L.lens_serve_sim.restype = vp
            L.lens_serve_submit.argtypes = [vp, ctypes.POINTER(LensRequest), ctypes.POINTER(ctypes.c_ulonglong)]
            L.lens_serve_wait.argtypes = [vp, ctypes.c_ulonglong, ip]
            L.lens_serve_poll.argtypes = [vp, ctypes.c_ulonglong]
            L.lens_serve_cancel.argtypes = [vp, ctypes.c_ulonglong]
            L.lens_serve_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_double)]
            L.lens_serve_pause.argtypes = [vp, ip]
            L.lens_serve_reset_stats.argtypes = [vp]
            L.lens_serve_destroy.argtypes = [vp]
            L.lens_serve_last_error.argtypes = [vp]
            L.lens_serve_last_error.restype = ctypes.c_char_p
            L.lens_serve_destroy.restype = None
            _lib = L
    return _lib


def _stream_ptr(stream: Optional[torch.cuda.Stream]) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        return int(t.data_ptr())
    return int(t.ctypes.data)


def profile_struct(name: str, params: Sequence[float], table=LENS_TYPES, cls=LensProfile):
    p = cls()
    p.type = table[name]
    for i, v in enumerate(params):
        p.p[i] = float(v)
    return p


class Simulator:
    """A lens_sim handle: resident PSFs and subhalo tables plus a device workspace."""

    def __init__(self, device: int = 0, mem_budget: int = 0, max_batch: int = 0):
        self._L = lib()
        cfg = SimConfig(device, mem_budget, max_batch, 0)
        h = ctypes.c_void_p()
        rc = self._L.lens_sim_create(ctypes.byref(cfg), ctypes.byref(h))
        if rc != 0:
            raise LensSimError(rc, "lens_sim_create failed")
        self.h = h
        self.device = device
        self._psf_ids: Dict[Tuple[int, bytes], int] = {}

    @classmethod
    def wrap(cls, handle: int, device: int = 0) -> "Simulator":
        """A non-owning view of an existing handle (e.g. a server's)."""
        obj = cls.__new__(cls)
        obj._L = lib()
        obj.h = ctypes.c_void_p(handle)
        obj.device = device
        obj._psf_ids = {}
        obj._borrowed = True
        return obj

    def close(self):
        if getattr(self, "h", None) is not None and not getattr(self, "_borrowed", False):
            self._L.lens_sim_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc: int):
        if rc != 0:
            raise LensSimError(rc, self._L.lens_sim_last_error(self.h).decode())

    def last_error(self) -> str:
        return self._L.lens_sim_last_error(self.h).decode()

    # ------------------------------------------------------------------ resident state
    def register_psf(self, kernel: np.ndarray) -> int:
        k = np.ascontiguousarray(kernel, dtype=np.float32)
        key = (k.shape[0], k.tobytes())
        if key in self._psf_ids:
            return self._psf_ids[key]
        pid = ctypes.c_int()
        self._check(self._L.lens_sim_register_psf(self.h, k.ctypes.data, int(k.shape[0]), ctypes.byref(pid)))
        self._psf_ids[key] = pid.value
        return pid.value

    def register_subhalos(self, soa) -> int:
        if isinstance(soa, torch.Tensor):
            t = soa.contiguous()
            n = int(t.shape[1]) if t.dim() == 2 else 0
            ptr = t.data_ptr() if n else None
        else:
            t = np.ascontiguousarray(soa, dtype=np.float32).reshape(5, -1)
            n = int(t.shape[1])
            ptr = t.ctypes.data if n else None
        tid = ctypes.c_int()
        self._check(self._L.lens_sim_register_subhalos(self.h, ptr, n, ctypes.byref(tid)))
        return tid.value

    # ------------------------------------------------------------------ marshalling
    def system_struct(self, system: W.LensSystem, keep: list, subhalos=None, subhalo_table: int = -1,
                      use_psf: bool = True) -> LensSystemC:
        g = system.grid
        c = LensSystemC()
        c.grid = LensGrid(int(g.nx), int(g.ny), int(g.s), float(g.dpix), float(g.x0), float(g.y0))
        nd = len(system.deflectors)
        arr = (LensProfile * max(nd, 1))()  # the library checks nd against LENS_MAX_DEFLECTORS
        for i, (name, vals) in enumerate(system.deflectors):
            arr[i] = profile_struct(name, vals)
        keep.append(arr)
        c.deflectors = ctypes.cast(arr, ctypes.POINTER(LensProfile))
        c.n_deflectors = nd
        if subhalo_table >= 0:
            c.subhalos = None
            c.n_subhalos = 0
            c.subhalo_table = subhalo_table
        else:
            src = subhalos if subhalos is not None else system.subhalos
            if isinstance(src, torch.Tensor):
                src = src.contiguous()
            else:
                src = np.ascontiguousarray(src, dtype=np.float32).reshape(5, -1)
            keep.append(src)
            n = int(src.shape[1])
            c.subhalos = _ptr(src) if n else None
            c.n_subhalos = n
            c.subhalo_table = -1
        c.source = profile_struct(system.source[0], system.source[1], LIGHT_TYPES, LightProfile)
        coef = getattr(system, "source_coeffs", None)
        if coef is not None:
            coef = np.ascontiguousarray(coef, dtype=np.float32).ravel()
            keep.append(coef)
            c.source_coeffs = coef.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
            c.n_source_coeffs = int(coef.size)
        c.psf_id = self.register_psf(system.psf) if (use_psf and system.psf is not None) else -1
        return c

    # ------------------------------------------------------------------ tuning
    def set_variant(self, variant: int) -> None:
        self._check(self._L.lens_sim_set_variant(self.h, int(variant)))

    def pipe_rates(self) -> dict:
        """Measured FP32 and MUFU rates of this GPU per SM and SM clock (lens_sim_pipe_rates):
        the denominators of the ALU-bound kernels' rooflines."""
        out = (ctypes.c_double * len(PIPE_RATES))()
        self._check(self._L.lens_sim_pipe_rates(self.h, out, len(PIPE_RATES)))
        return {k: float(v) for k, v in zip(PIPE_RATES, out)}

    def set_far_field(self, kappa: float) -> None:
        """Far-field interpolation of the subhalo sum for image calls (0: the exact sum, the
        default; >= 3: subhalos kappa box half-widths from a work unit are summed at 8 x 8
        Chebyshev nodes and interpolated -- changes results within the bound the C header
        states)."""
        self._check(self._L.lens_sim_set_far_field(self.h, float(kappa)))
        self.far_kappa = float(kappa)

    def set_conv_method(self, method: str) -> None:
        """PSF method: "auto" (FFT for k >= 33 when it fits), "direct" or "fft"."""
        self._check(self._L.lens_sim_set_conv_method(self.h, CONV_METHODS[method]))

    def autotune(self, system: W.LensSystem, reps: int = 5, use_cache: bool = True, stream=None):
        """Pick the fastest trace-kernel launch variant for systems shaped like `system`.

        Results are cached per GPU name and shape bucket (grid, supersampling, subhalo count
        rounded to a power of two) in _build/autotune.json."""
        import json
        g = system.grid
        nsub = system.n_sub
        bucket = f"{g.nx}x{g.ny}/s{g.s}/sub{1 << max(nsub, 1).bit_length()}"
        if getattr(self, "far_kappa", 0.0) > 0.0:
            bucket += f"/far{self.far_kappa:g}"
        key = f"{torch.cuda.get_device_name(self.device)}|{bucket}"
        cache = {}
        if use_cache and os.path.exists(_TUNE_CACHE):
            try:
                cache = json.load(open(_TUNE_CACHE))
            except (OSError, ValueError):
                cache = {}
        if use_cache and key in cache:
            self.set_variant(cache[key]["variant"])
            return cache[key]
        keep: list = []
        c = self.system_struct(system, keep, use_psf=False)
        best = ctypes.c_int()
        ms = (ctypes.c_float * len(TRACE_VARIANTS))()
        self._check(self._L.lens_sim_autotune(self.h, ctypes.byref(c), int(reps), ctypes.byref(best), ms,
                                              len(TRACE_VARIANTS), _stream_ptr(stream)))
        entry = {"variant": best.value, "name": TRACE_VARIANTS[best.value],
                 "ms": {TRACE_VARIANTS[i]: float(ms[i]) for i in range(len(TRACE_VARIANTS))}}
        if use_cache:
            cache[key] = entry
            os.makedirs(os.path.dirname(_TUNE_CACHE), exist_ok=True)
            tmp = _TUNE_CACHE + f".tmp{os.getpid()}"
            with open(tmp, "w") as fh:
                json.dump(cache, fh, indent=1)
            os.replace(tmp, _TUNE_CACHE)
        return entry

    def set_batch_schedule(self, form: int, order: int = 0) -> None:
        """Persistent trace kernel form (BATCH_FORMS index) and unit-queue order of batched calls."""
        self._check(self._L.lens_sim_set_batch_schedule(self.h, int(form), int(order)))

    def autotune_batch(self, systems, out: Optional[List] = None, reps: int = 3, use_cache: bool = True,
                       stream=None):
        """Pick the fastest schedule of the batched launch for batches shaped like `systems`.

        Results are cached per GPU name and batch bucket (system count and mean pair count, each
        rounded to a power of two, the largest grid and supersampling) in _build/autotune.json."""
        import json
        n = len(systems)
        pairs = sum(s_.pairs() for s_ in systems) / max(n, 1)
        bucket = (f"batch/n{1 << max(n, 1).bit_length()}/pairs{1 << int(max(pairs, 1)).bit_length()}"
                  f"/nx{max(s_.grid.nx for s_ in systems)}/s{max(s_.grid.s for s_ in systems)}")
        key = f"{torch.cuda.get_device_name(self.device)}|{bucket}"
        cache = {}
        if use_cache and os.path.exists(_TUNE_CACHE):
            try:
                cache = json.load(open(_TUNE_CACHE))
            except (OSError, ValueError):
                cache = {}
        if use_cache and key in cache:
            self.set_batch_schedule(cache[key]["form"], cache[key]["order"])
            return cache[key]
        keep: list = []
        arr = (LensSystemC * n)()
        for i, s_ in enumerate(systems):
            arr[i] = self.system_struct(s_, keep)
        if out is None:
            out = [torch.empty((s_.grid.ny, s_.grid.nx), dtype=torch.float32, device=f"cuda:{self.device}")
                   for s_ in systems]
        ptrs = (ctypes.c_void_p * n)(*[_ptr(o) for o in out])
        bf, bo = ctypes.c_int(), ctypes.c_int()
        ms = (ctypes.c_float * (2 * len(BATCH_FORMS)))()
        self._check(self._L.lens_sim_autotune_batch(self.h, arr, n, ptrs, int(reps), ctypes.byref(bf),
                                                    ctypes.byref(bo), ms, _stream_ptr(stream)))
        entry = {"form": bf.value, "order": bo.value,
                 "name": f"{BATCH_FORMS[bf.value]}/{BATCH_ORDERS[bo.value]}",
                 "ms": {f"{BATCH_FORMS[f]}/{BATCH_ORDERS[o]}": float(ms[2 * f + o])
                        for f in range(len(BATCH_FORMS)) for o in range(2)}}
        if use_cache:
            cache[key] = entry
            os.makedirs(os.path.dirname(_TUNE_CACHE), exist_ok=True)
            tmp = _TUNE_CACHE + f".tmp{os.getpid()}"
            with open(tmp, "w") as fh:
                json.dump(cache, fh, indent=1)
            os.replace(tmp, _TUNE_CACHE)
        return entry

    # ------------------------------------------------------------------ compute
    def image(self, systems, out: Optional[List] = None, stream=None, subhalos=None, subhalo_tables=None,
              use_psf: bool = True) -> List[torch.Tensor]:
        """Simulate images.  `out` may hold CUDA tensors or NumPy arrays (host outputs)."""
        if isinstance(systems, W.LensSystem):
            systems = [systems]
        n = len(systems)
        keep: list = []
        arr = (LensSystemC * n)()
        for i, s in enumerate(systems):
            arr[i] = self.system_struct(s, keep, None if subhalos is None else subhalos[i],
                                        -1 if subhalo_tables is None else subhalo_tables[i], use_psf)
        if out is None:
            out = [torch.empty((s.grid.ny, s.grid.nx), dtype=torch.float32, device=f"cuda:{self.device}")
                   for s in systems]
        ptrs = (ctypes.c_void_p * n)(*[_ptr(o) for o in out])
        self._check(self._L.lens_sim_image(self.h, arr, n, ptrs, _stream_ptr(stream)))
        return out

    def deflection(self, system: W.LensSystem, x: torch.Tensor, y: torch.Tensor, stream=None):
        keep: list = []
        c = self.system_struct(system, keep, use_psf=False)
        x = x.contiguous().float()
        y = y.contiguous().float()
        ax = torch.empty_like(x)
        ay = torch.empty_like(y)
        self._check(self._L.lens_sim_deflection(self.h, ctypes.byref(c), x.data_ptr(), y.data_ptr(), x.numel(),
                                                ax.data_ptr(), ay.data_ptr(), _stream_ptr(stream)))
        return ax, ay

    def convolve(self, images: torch.Tensor, psf, out: Optional[torch.Tensor] = None, stream=None):
        pid = psf if isinstance(psf, int) else self.register_psf(psf)
        imgs = images.contiguous()
        if imgs.dim() == 2:
            imgs = imgs[None]
        if out is None:
            out = torch.empty_like(imgs)
        self._check(self._L.lens_sim_convolve(self.h, imgs.data_ptr(), imgs.shape[0], imgs.shape[1],
                                              imgs.shape[2], pid, out.data_ptr(), _stream_ptr(stream)))
        return out

    def grad(self, system: W.LensSystem, data: torch.Tensor, sigma_bkg: float, t_exp: float,
             params: torch.Tensor, want_grad: bool = True, stream=None, subhalo_table: int = -1):
        keep: list = []
        c = self.system_struct(system, keep, subhalo_table=subhalo_table)
        P = params.contiguous().float()
        n = P.shape[0]
        L = torch.empty(n, dtype=torch.float32, device=P.device)
        G = torch.empty((n, 15), dtype=torch.float32, device=P.device) if want_grad else None
        self._check(self._L.lens_sim_grad(self.h, ctypes.byref(c), data.contiguous().data_ptr(), float(sigma_bkg),
                                          float(t_exp), P.data_ptr(), n, L.data_ptr(),
                                          None if G is None else G.data_ptr(), _stream_ptr(stream)))
        return (L, G) if want_grad else L


def _linear_amp(self, system: W.LensSystem, data: torch.Tensor, sigma_bkg: float, t_exp: float,
                params: torch.Tensor, stream=None, subhalo_table: int = -1):
    """Weighted least-squares source amplitude (and logL at it) for [n, 15] parameter points."""
    keep: list = []
    c = self.system_struct(system, keep, subhalo_table=subhalo_table)
    P = params.contiguous().float()
    n = P.shape[0]
    amp = torch.empty(n, dtype=torch.float32, device=P.device)
    L = torch.empty(n, dtype=torch.float32, device=P.device)
    self._check(self._L.lens_sim_linear_amp(self.h, ctypes.byref(c), data.contiguous().data_ptr(), float(sigma_bkg),
                                            float(t_exp), P.data_ptr(), n, amp.data_ptr(), L.data_ptr(),
                                            _stream_ptr(stream)))
    return amp, L


Simulator.linear_amp = _linear_amp


class LensLogLike(torch.autograd.Function):
    """chi^2 log-likelihood of [n, 15] parameter points as an autograd op.

    forward runs lens_sim_grad once (likelihood and the hand-written adjoint together) and
    keeps the gradient; backward scales it by the incoming gradient.
    """

    @staticmethod
    def forward(ctx, params, sim, system, data, sigma_bkg, t_exp, subhalo_table=-1):
        L, G = sim.grad(system, data, sigma_bkg, t_exp, params.detach(), want_grad=True,
                        subhalo_table=subhalo_table)
        ctx.save_for_backward(G)
        return L

    @staticmethod
    def backward(ctx, grad_L):
        (G,) = ctx.saved_tensors
        return grad_L[:, None] * G, None, None, None, None, None, None


class Server:
    """A lens_server: continuous batching of image and likelihood+gradient requests.

    Requests reference host NumPy buffers, which must stay alive until wait()/poll() reports
    the request finished; the server keeps them referenced until then."""

    def __init__(self, device: int = 0, max_inflight: int = 4096, mem_budget: int = 0):
        self._L = lib()
        cfg = SimConfig(device, mem_budget, 0, 0)
        h = ctypes.c_void_p()
        rc = self._L.lens_serve_create(ctypes.byref(cfg), int(max_inflight), ctypes.byref(h))
        if rc != 0:
            raise LensSimError(rc, "lens_serve_create failed")
        self.h = h
        self.sim = Simulator.wrap(self._L.lens_serve_sim(h), device)
        self._keep: Dict[int, list] = {}

    def close(self):
        if getattr(self, "h", None) is not None:
            self._L.lens_serve_destroy(self.h)
            self.h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit_image(self, system: W.LensSystem, out: np.ndarray) -> int:
        return self.submit_prepared(self.prepare_image(system, out))

    def submit_loglike(self, system: W.LensSystem, data: np.ndarray, sigma_bkg: float, t_exp: float,
                       params: np.ndarray, out: np.ndarray, out_grad: Optional[np.ndarray]) -> int:
        return self.submit_prepared(self.prepare_loglike(system, data, sigma_bkg, t_exp, params, out, out_grad))

    def prepare_image(self, system: W.LensSystem, out: np.ndarray):
        """The marshalled request (struct and the objects it points into), for submit_prepared."""
        keep: list = [out]
        req = LensRequest()
        req.kind = 0
        req.sys = self.sim.system_struct(system, keep)
        req.out = out.ctypes.data
        keep.append(req)
        return req, keep

    def prepare_loglike(self, system: W.LensSystem, data: np.ndarray, sigma_bkg: float, t_exp: float,
                        params: np.ndarray, out: np.ndarray, out_grad: Optional[np.ndarray]):
        data = np.ascontiguousarray(data, np.float32)
        params = np.ascontiguousarray(params, np.float32)
        keep: list = [data, params, out, out_grad]
        req = LensRequest()
        req.kind = 1
        req.sys = self.sim.system_struct(system, keep)
        req.data = data.ctypes.data
        req.sigma_bkg = float(sigma_bkg)
        req.t_exp = float(t_exp)
        req.params = params.ctypes.data
        req.out = out.ctypes.data
        req.out_grad = None if out_grad is None else out_grad.ctypes.data
        keep.append(req)
        return req, keep

    def submit_prepared(self, prepared) -> int:
        """Submit a request from prepare_image / prepare_loglike; the buffers it references must
        stay alive (the server keeps them referenced until wait/poll reports the result)."""
        req, keep = prepared
        t = ctypes.c_ulonglong()
        rc = self._L.lens_serve_submit(self.h, ctypes.byref(req), ctypes.byref(t))
        if rc != 0:
            raise LensSimError(rc, "lens_serve_submit")
        self._keep[t.value] = keep
        return t.value

    def last_error(self) -> str:
        """Text of the server's most recent failed request ("" if none)."""
        return (self._L.lens_serve_last_error(self.h) or b"").decode()

    def wait(self, ticket: int, timeout_ms: int = 60000) -> int:
        rc = self._L.lens_serve_wait(self.h, ticket, int(timeout_ms))
        if rc != LENS_ERR_TIMEOUT:
            self._keep.pop(ticket, None)
        return rc

    def poll(self, ticket: int) -> int:
        rc = self._L.lens_serve_poll(self.h, ticket)
        if rc != LENS_ERR_BUSY:
            self._keep.pop(ticket, None)
        return rc

    def cancel(self, ticket: int) -> int:
        return self._L.lens_serve_cancel(self.h, ticket)

    def pause(self, paused: bool = True) -> None:
        self._L.lens_serve_pause(self.h, 1 if paused else 0)

    def stats(self):
        a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        self._L.lens_serve_stats(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
        return {"p50_ms": a.value, "p99_ms": b.value, "requests_per_s": c.value}

    def reset_stats(self) -> None:
        self._L.lens_serve_reset_stats(self.h)

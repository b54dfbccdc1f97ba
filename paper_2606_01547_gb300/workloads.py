"""Seeded synthetic inputs shaped like the paper's image-simulation workloads.

This module only draws inputs: grid specs, deflector and source parameters, subhalo
populations, sampled PSF kernels and observation noise.  It holds none of the
lensing arithmetic, and it is the one module that both the CUDA path (through the
binding) and the FP64 oracle (through the tests) read.  Every parameter is drawn in
FP64 from a NumPy ``Generator(PCG64(seed))`` and rounded to FP32, and the same FP32
values feed both sides, so parameter rounding is not a parity question.

Profile names follow the deflector and light tables of the paper (EPL, NIE/SIE,
SHEAR, SIS, NFW, TNFW; SERSIC, SERSIC_ELLIPSE, SERSIC_ELLIPSE_Q_PHI).  Parameter
layouts (angles in arcsec, position angles in radians):

=====================  ==========================================
SIS                    theta_E, cx, cy
SIE                    theta_E, q, phi, cx, cy
SIE_E1E2               theta_E, e1, e2, cx, cy
EPL                    theta_E, gamma, q, phi, cx, cy
EPL_E1E2               theta_E, gamma, e1, e2, cx, cy
SHEAR                  gamma1, gamma2
POINT_MASS             theta_E, cx, cy
NFW                    Rs, alpha_Rs, cx, cy
TNFW                   Rs, alpha_Rs, r_t, cx, cy
SERSIC_ELLIPSE_Q_PHI   amp, R_sersic, n, q, phi, cx, cy
SERSIC_ELLIPSE         amp, R_sersic, n, e1, e2, cx, cy
SERSIC                 amp, R_sersic, n, cx, cy
=====================  ==========================================

Subhalos are a float32 structure-of-arrays ``[5, n]``: cx, cy, Rs, alpha_Rs, r_t.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

LENS_NAMES = ("SIS", "SIE", "EPL", "SHEAR", "POINT_MASS", "NFW", "TNFW", "EPL_E1E2", "SIE_E1E2")
LIGHT_NAMES = ("SERSIC_ELLIPSE_Q_PHI", "SERSIC_ELLIPSE", "SERSIC")
N_PARAMS = {"SIS": 3, "SIE": 5, "EPL": 6, "SHEAR": 2, "POINT_MASS": 3, "NFW": 4, "TNFW": 5,
            "EPL_E1E2": 6, "SIE_E1E2": 5, "MULTIPOLE": 6, "EPL_MULTIPOLE_M1M3M4": 12, "CSE": 6,
            "NFW_ELLIPSE_CSE": 6, "HERNQUIST_ELLIPSE_CSE": 6, "MULTIPOLE_ELL": 8,
            "SERSIC_ELLIPSE_Q_PHI": 7, "SERSIC_ELLIPSE": 7, "SERSIC": 5, "SHAPELETS": 4}
# Order of the 15 free parameters of the likelihood (differentiation workload).
FREE_PARAMS = ("epl_theta_E", "epl_gamma", "epl_e1", "epl_e2", "epl_cx", "epl_cy",
               "shear_g1", "shear_g2",
               "src_amp", "src_R", "src_n", "src_e1", "src_e2", "src_cx", "src_cy")


def f32(v) -> float:
    """Round to the nearest FP32 value, returned as a Python float."""
    return float(np.float32(v))


@dataclasses.dataclass
class Grid:
    nx: int
    ny: int
    s: int          # supersampling factor
    dpix: float     # pixel scale, arcsec
    x0: float = 0.0  # grid centre, arcsec
    y0: float = 0.0


@dataclasses.dataclass
class LensSystem:
    grid: Grid
    deflectors: List[Tuple[str, List[float]]]
    subhalos: np.ndarray                        # float32 [5, n]
    source: Tuple[str, List[float]]
    psf: Optional[np.ndarray] = None            # float32 [k, k], k odd, or None
    source_coeffs: Optional[np.ndarray] = None  # float32 SHAPELETS amplitudes, else None

    @property
    def n_sub(self) -> int:
        return int(self.subhalos.shape[1])

    def pairs(self) -> int:
        """Point-subhalo pairs of the subhalo sum (the dominant work)."""
        g = self.grid
        return g.nx * g.ny * g.s * g.s * self.n_sub


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _profile(name: str, vals: Sequence[float]) -> Tuple[str, List[float]]:
    assert len(vals) == N_PARAMS[name], name
    return name, [f32(v) for v in vals]


# ----------------------------------------------------------------------------- PSF kernels
def gaussian_psf(fwhm: float, dpix: float, k: int) -> np.ndarray:
    """Gaussian PSF sampled at pixel centres on a k x k grid and normalised (FP64 -> FP32)."""
    assert k % 2 == 1
    sigma = fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0))) / dpix
    c = (k - 1) / 2
    yy, xx = np.mgrid[0:k, 0:k].astype(np.float64) - c
    ker = np.exp(-(xx * xx + yy * yy) / (2.0 * sigma * sigma))
    return (ker / ker.sum()).astype(np.float32)


def moffat_psf(beta: float, fwhm: float, dpix: float, k: int) -> np.ndarray:
    """Moffat PSF (1 + r^2/a^2)^-beta, a = FWHM / (2 sqrt(2^(1/beta) - 1)), sampled and normalised."""
    assert k % 2 == 1
    a = fwhm / (2.0 * math.sqrt(2.0 ** (1.0 / beta) - 1.0)) / dpix
    c = (k - 1) / 2
    yy, xx = np.mgrid[0:k, 0:k].astype(np.float64) - c
    ker = (1.0 + (xx * xx + yy * yy) / (a * a)) ** (-beta)
    return (ker / ker.sum()).astype(np.float32)


# ----------------------------------------------------------------------------- draws
def _qphi_to_e(q: float, phi: float) -> Tuple[float, float]:
    """Ellipticity components for an axis ratio and angle (input drawing only)."""
    c = (1.0 - q) / (1.0 + q)
    return c * math.cos(2.0 * phi), c * math.sin(2.0 * phi)


def subhalo_population(rng: np.random.Generator, n: int, radius: float = 3.0) -> np.ndarray:
    """n truncated-NFW subhalos: positions uniform in a disc of the given radius,
    Rs log-uniform in [0.005, 0.05]", alpha_Rs log-uniform in [1e-4, 1e-2]", r_t = 5 Rs."""
    u = rng.random(n)
    ang = rng.random(n) * 2.0 * math.pi
    r = radius * np.sqrt(u)
    rs = np.exp(rng.uniform(math.log(0.005), math.log(0.05), n))
    ars = np.exp(rng.uniform(math.log(1e-4), math.log(1e-2), n))
    soa = np.stack([r * np.cos(ang), r * np.sin(ang), rs, ars, 5.0 * rs])
    return soa.astype(np.float32)


def log_uniform_count(rng: np.random.Generator, hi: int = 20000) -> int:
    """Subhalo count 'log-uniform in [0, hi]': floor(exp(U[0, ln(hi+1)])) - 1."""
    return int(math.floor(math.exp(rng.uniform(0.0, math.log(hi + 1.0))))) - 1


def _main_and_shear(rng: np.random.Generator):
    theta_e = rng.uniform(0.8, 1.4)
    gamma = rng.uniform(1.8, 2.2)
    q = rng.uniform(0.6, 0.95)
    phi = rng.uniform(0.0, math.pi)
    gmag = rng.uniform(0.0, 0.08)
    gang = rng.uniform(0.0, math.pi)
    return (_profile("EPL", [theta_e, gamma, q, phi, 0.0, 0.0]),
            _profile("SHEAR", [gmag * math.cos(2 * gang), gmag * math.sin(2 * gang)]))


def _sersic_q_phi(rng: np.random.Generator):
    n = rng.uniform(0.5, 4.0)
    r = rng.uniform(0.05, 0.5)
    q = rng.uniform(0.6, 0.95)
    phi = rng.uniform(0.0, math.pi)
    cx, cy = rng.uniform(-0.1, 0.1, 2)
    return _profile("SERSIC_ELLIPSE_Q_PHI", [10.0, r, n, q, phi, cx, cy])


def plain_system() -> LensSystem:
    """60x60 grid at 0.05", no supersampling; SIE (theta_E=1, q=0.8, phi=0.3) + shear
    (0.03, -0.02); Sersic (amp 10, R 0.2", n 1.5, q 0.7, centre (0.05, -0.03));
    5x5 Gaussian PSF with FWHM 0.1"."""
    return LensSystem(
        grid=Grid(60, 60, 1, f32(0.05)),
        deflectors=[_profile("SIE", [1.0, 0.8, 0.3, 0.0, 0.0]), _profile("SHEAR", [0.03, -0.02])],
        subhalos=np.zeros((5, 0), np.float32),
        source=_profile("SERSIC_ELLIPSE_Q_PHI", [10.0, 0.2, 1.5, 0.7, 0.0, 0.05, -0.03]),
        psf=gaussian_psf(0.1, 0.05, 5),
    )


def substructure_system(seed: int, n_sub: int = 10000, nx: int = 200, s: int = 3,
                        dpix: float = 0.04, k: int = 21) -> LensSystem:
    """200x200 grid at 0.04", supersampling 3; EPL + shear; 10,000 TNFW subhalos in a 3"
    disc; elliptical Sersic; 21x21 Moffat PSF (beta 3, FWHM 0.12")."""
    rng = _rng(seed)
    epl, shear = _main_and_shear(rng)
    src = _sersic_q_phi(rng)
    sub = subhalo_population(rng, n_sub)
    return LensSystem(Grid(nx, nx, s, f32(dpix)), [epl, shear], sub, src,
                      moffat_psf(3.0, 0.12, dpix, k) if k > 0 else None)


def multipole_shapelet_system(seed: int, n_max: int = 6, n_sub: int = 1000, nx: int = 60, s: int = 2,
                              dpix: float = 0.05, k: int = 5) -> LensSystem:
    """Profile-variant workload: EPL_MULTIPOLE_M1M3M4 (EPL as the substructure workload plus
    m = 1, 3, 4 multipoles with a_m ~ U[0, 0.02], dphi_m ~ U[0, pi)) + shear + TNFW subhalos,
    and a SHAPELETS source (beta ~ U[0.08, 0.2]", centre ~ U[-0.1, 0.1]", amplitudes
    N(0, 1) / (1 + n1 + n2) plus 3 on the (0, 0) mode); Gaussian PSF (FWHM 0.1")."""
    rng = _rng(seed)
    epl, shear = _main_and_shear(rng)
    th, g, q, phi, cx, cy = epl[1]
    c = (1.0 - q) / (1.0 + q)
    e1, e2 = c * math.cos(2.0 * phi), c * math.sin(2.0 * phi)
    mult = [v for _ in range(3) for v in (rng.uniform(0.0, 0.02), rng.uniform(0.0, math.pi))]
    lens = _profile("EPL_MULTIPOLE_M1M3M4", [th, g, e1, e2, cx, cy] + mult)
    sub = subhalo_population(rng, n_sub)
    beta = rng.uniform(0.08, 0.2)
    src = _profile("SHAPELETS", [n_max, beta, rng.uniform(-0.1, 0.1), rng.uniform(-0.1, 0.1)])
    idx = [(n1, n - n1) for n in range(n_max + 1) for n1 in range(n, -1, -1)]
    coeffs = np.array([rng.normal() / (1.0 + n1 + n2) for n1, n2 in idx])
    coeffs[0] += 3.0
    return LensSystem(Grid(nx, nx, s, f32(dpix)), [lens, shear], sub, src,
                      gaussian_psf(0.1, dpix, k) if k > 0 else None, coeffs.astype(np.float32))


BATCH_GRIDS = (64, 100, 128, 200, 256)
BATCH_SUPERSAMPLE = (1, 2, 3)
BATCH_PSF = tuple(range(5, 32, 2))


def batched_systems(seed: int, count: int = 4096, max_sub: int = 20000,
                    grids: Sequence[int] = BATCH_GRIDS) -> List[LensSystem]:
    """Uneven batch: grid from {64,100,128,200,256}^2, s in {1,2,3}, subhalo count
    log-uniform in [0, 20000], parameters as the substructure workload, PSF 5x5..31x31."""
    rng = _rng(seed)
    out = []
    for _ in range(count):
        nx = int(rng.choice(grids))
        s = int(rng.choice(BATCH_SUPERSAMPLE))
        k = int(rng.choice(BATCH_PSF))
        nsub = log_uniform_count(rng, max_sub)
        epl, shear = _main_and_shear(rng)
        src = _sersic_q_phi(rng)
        sub = subhalo_population(rng, nsub)
        out.append(LensSystem(Grid(nx, nx, s, f32(0.04)), [epl, shear], sub, src,
                              moffat_psf(3.0, 0.12, 0.04, k)))
    return out


@dataclasses.dataclass
class DiffProblem:
    system: LensSystem          # truth model (EPL_E1E2 + SHEAR, SERSIC_ELLIPSE, fixed subhalos)
    truth: np.ndarray           # float32 [15]
    points: np.ndarray          # float32 [n_points, 15]
    sigma_bkg: float
    t_exp: float


def _draw_free(rng: np.random.Generator) -> List[float]:
    theta_e = rng.uniform(0.8, 1.4)
    gamma = rng.uniform(1.8, 2.2)
    e1, e2 = _qphi_to_e(rng.uniform(0.6, 0.95), rng.uniform(0.0, math.pi))
    ecx, ecy = rng.uniform(-0.05, 0.05, 2)
    gmag = rng.uniform(0.0, 0.08)
    gang = rng.uniform(0.0, math.pi)
    amp = rng.uniform(5.0, 15.0)
    r = rng.uniform(0.05, 0.5)
    n = rng.uniform(0.5, 4.0)
    se1, se2 = _qphi_to_e(rng.uniform(0.6, 0.95), rng.uniform(0.0, math.pi))
    scx, scy = rng.uniform(-0.1, 0.1, 2)
    return [theta_e, gamma, e1, e2, ecx, ecy, gmag * math.cos(2 * gang), gmag * math.sin(2 * gang),
            amp, r, n, se1, se2, scx, scy]


def system_from_free(base: LensSystem, p: Sequence[float]) -> LensSystem:
    """The base system with its EPL_E1E2, SHEAR and SERSIC_ELLIPSE set from a 15-vector."""
    return LensSystem(base.grid,
                      [_profile("EPL_E1E2", p[0:6]), _profile("SHEAR", p[6:8])],
                      base.subhalos,
                      _profile("SERSIC_ELLIPSE", p[8:15]),
                      base.psf)


def diff_problem(seed: int, n_points: int = 512, n_sub: int = 1000, nx: int = 100,
                 dpix: float = 0.05, k: int = 13) -> DiffProblem:
    """100x100 grid at 0.05" (s=1), EPL + shear + elliptical Sersic with 15 free
    parameters, 1,000 fixed TNFW subhalos, 13x13 Gaussian PSF (FWHM 0.1"), sigma_bkg 0.01,
    t_exp 1000 s, and n_points parameter vectors drawn from the priors."""
    rng = _rng(seed)
    truth = np.array(_draw_free(rng), np.float32)
    sub = subhalo_population(rng, n_sub)
    pts = np.array([_draw_free(rng) for _ in range(n_points)], np.float32).reshape(n_points, 15)
    base = LensSystem(Grid(nx, nx, 1, f32(dpix)), [], sub, ("SERSIC_ELLIPSE", [0.0] * 7),
                      gaussian_psf(0.1, dpix, k))
    return DiffProblem(system_from_free(base, truth), truth, pts, 0.01, 1000.0)


def observe(model: np.ndarray, sigma_bkg: float, t_exp: float, seed: int) -> np.ndarray:
    """Synthetic observation: model + N(0, sigma_bkg^2) + Poisson(max(m,0) t_exp)/t_exp - max(m,0),
    drawn in FP64 and rounded to FP32."""
    rng = _rng(seed)
    m = np.asarray(model, np.float64)
    mp = np.maximum(m, 0.0)
    d = m + rng.normal(0.0, sigma_bkg, m.shape) + (rng.poisson(mp * t_exp) / t_exp - mp)
    return d.astype(np.float32)


@dataclasses.dataclass
class Request:
    t_arrival: float            # seconds from stream start
    kind: int                   # 0 image, 1 log-likelihood + gradient
    system: LensSystem


def serving_stream(seed: int, rate: float, duration: float, image_frac: float = 0.7,
                   max_sub: int = 20000) -> List[Request]:
    """Open-loop Poisson arrivals; 70% image / 30% likelihood+gradient; grids 64..256 (even),
    subhalos log-uniform in [0, 20000], PSF 5x5..31x31 (odd)."""
    rng = _rng(seed)
    t = 0.0
    out = []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        kind = 0 if rng.random() < image_frac else 1
        nx = int(rng.integers(32, 129)) * 2
        k = int(rng.choice(BATCH_PSF))
        nsub = log_uniform_count(rng, max_sub)
        if kind == 0:
            epl, shear = _main_and_shear(rng)
            src = _sersic_q_phi(rng)
            sysm = LensSystem(Grid(nx, nx, 1, f32(0.04)), [epl, shear], subhalo_population(rng, nsub),
                              src, moffat_psf(3.0, 0.12, 0.04, k))
        else:
            p = _draw_free(rng)
            base = LensSystem(Grid(nx, nx, 1, f32(0.04)), [], subhalo_population(rng, nsub),
                              ("SERSIC_ELLIPSE", [0.0] * 7), moffat_psf(3.0, 0.12, 0.04, k))
            sysm = system_from_free(base, p)
        out.append(Request(t, kind, sysm))
    return out

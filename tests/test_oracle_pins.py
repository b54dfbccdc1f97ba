"""Pins of the FP64 oracle against what the physics and mathematics fix.

None of these checks re-types an oracle formula.  Each compares the oracle with an
independent route: quadrature of a 3-D density, the Schramm/Keeton 1-D integral for
elliptical mass, finite-difference divergence against the convergence definition,
SciPy's convolution, the Sersic closed-form flux, a pixel-area quadrature, and central
finite differences of the likelihood.
"""
import math

import numpy as np
import pytest
from scipy import integrate, signal, special

import oracle
from paper_2606_01547_gb300 import workloads as W

LN2 = math.log(2.0)


def _pts(n, seed, lo=-2.0, hi=2.0):
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, n), rng.uniform(lo, hi, n)


def _fd_div_curl(name, p, x, y, h):
    axp, _ = oracle.alpha(name, p, x + h, y)
    axm, _ = oracle.alpha(name, p, x - h, y)
    _, ayp = oracle.alpha(name, p, x, y + h)
    _, aym = oracle.alpha(name, p, x, y - h)
    _, ay_xp = oracle.alpha(name, p, x + h, y)
    _, ay_xm = oracle.alpha(name, p, x - h, y)
    ax_yp, _ = oracle.alpha(name, p, x, y + h)
    ax_ym, _ = oracle.alpha(name, p, x, y - h)
    div = (axp - axm) / (2 * h) + (ayp - aym) / (2 * h)
    curl = (ay_xp - ay_xm) / (2 * h) - (ax_yp - ax_ym) / (2 * h)
    return div, curl


def _ell_frame(x, y, phi, cx, cy):
    dx, dy = x - cx, y - cy
    return math.cos(phi) * dx + math.sin(phi) * dy, -math.sin(phi) * dx + math.cos(phi) * dy


# ----------------------------------------------------------------------------- point-like profiles
def test_sis_deflection_magnitude_is_theta_e():
    x, y = _pts(500, 1)
    ax, ay = oracle.alpha("SIS", [1.3, 0.1, -0.2], x, y)
    np.testing.assert_allclose(np.hypot(ax, ay), 1.3, rtol=1e-14)
    # radial direction: alpha parallel to (x - c)
    cross = ax * (y + 0.2) - ay * (x - 0.1)
    assert np.abs(cross).max() < 1e-13


def test_point_mass_gauss_law_and_zero_convergence():
    x, y = _pts(300, 2)
    ax, ay = oracle.alpha("POINT_MASS", [0.7, -0.3, 0.2], x, y)
    r = np.hypot(x + 0.3, y - 0.2)
    # enclosed mass: |alpha| r = theta_E^2, independent of r
    np.testing.assert_allclose(np.hypot(ax, ay) * r, 0.49, rtol=1e-14)
    keep = r > 0.2
    div, curl = _fd_div_curl("POINT_MASS", [0.7, -0.3, 0.2], x[keep], y[keep], 1e-5)
    assert np.abs(div).max() < 1e-4 and np.abs(curl).max() < 1e-4


def test_shear_is_traceless_and_curl_free():
    x, y = _pts(100, 3)
    div, curl = _fd_div_curl("SHEAR", [0.05, -0.03], x, y, 1e-4)
    assert np.abs(div).max() < 1e-10 and np.abs(curl).max() < 1e-10
    # the Jacobian's traceless part is the shear: d ax/dx = g1, d ax/dy = g2
    ax1, _ = oracle.alpha("SHEAR", [0.05, -0.03], [1.0], [0.0])
    ax2, _ = oracle.alpha("SHEAR", [0.05, -0.03], [0.0], [1.0])
    assert abs(ax1[0] - 0.05) < 1e-15 and abs(ax2[0] + 0.03) < 1e-15


# ----------------------------------------------------------------------------- SIE / EPL
def _kappa_epl(x, y, theta_e, gamma, q, phi, cx, cy):
    xp, yp = _ell_frame(x, y, phi, cx, cy)
    return (3.0 - gamma) / 2.0 * (theta_e / np.sqrt(q * xp * xp + yp * yp / q)) ** (gamma - 1.0)


@pytest.mark.parametrize("q,phi", [(0.8, 0.3), (0.55, 2.2), (0.95, -0.7)])
def test_sie_divergence_is_twice_kappa(q, phi):
    x, y = _pts(200, 4)
    p = [1.1, q, phi, 0.05, -0.1]
    keep = np.hypot(x - 0.05, y + 0.1) > 0.1
    x, y = x[keep], y[keep]
    div, curl = _fd_div_curl("SIE", p, x, y, 1e-5)
    kap = _kappa_epl(x, y, 1.1, 2.0, q, phi, 0.05, -0.1)
    np.testing.assert_allclose(div, 2 * kap, rtol=1e-6, atol=1e-8)
    assert np.abs(curl).max() < 1e-6


def test_sie_round_limit_is_sis():
    x, y = _pts(100, 5)
    a = oracle.alpha("SIE", [0.9, 1.0 - 1e-9, 0.4, 0.0, 0.0], x, y)
    b = oracle.alpha("SIS", [0.9, 0.0, 0.0], x, y)
    np.testing.assert_allclose(a[0], b[0], atol=1e-8)
    np.testing.assert_allclose(a[1], b[1], atol=1e-8)


@pytest.mark.parametrize("q,phi", [(0.8, 0.3), (0.6, 1.9), (0.3, -0.4)])
def test_epl_at_gamma2_equals_sie(q, phi):
    x, y = _pts(400, 6)
    a = oracle.alpha("EPL", [1.2, 2.0, q, phi, 0.1, 0.02], x, y)
    b = oracle.alpha("SIE", [1.2, q, phi, 0.1, 0.02], x, y)
    np.testing.assert_allclose(a[0], b[0], rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(a[1], b[1], rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("gamma,q,phi", [(1.8, 0.7, 0.2), (2.2, 0.6, 1.3), (2.05, 0.9, 2.9)])
def test_epl_divergence_is_twice_kappa(gamma, q, phi):
    x, y = _pts(200, 7)
    keep = np.hypot(x, y) > 0.1
    x, y = x[keep], y[keep]
    p = [1.0, gamma, q, phi, 0.0, 0.0]
    div, curl = _fd_div_curl("EPL", p, x, y, 1e-5)
    np.testing.assert_allclose(div, 2 * _kappa_epl(x, y, *p), rtol=1e-6, atol=1e-8)
    assert np.abs(curl).max() < 1e-6


def test_epl_round_closed_form():
    # q = 1: |alpha| = theta_E^(gamma-1) r^(2-gamma) (mass inside a circle of radius r)
    x, y = _pts(100, 8)
    for gamma in (1.7, 2.0, 2.3):
        ax, ay = oracle.alpha("EPL", [1.3, gamma, 1.0, 0.0, 0.0, 0.0], x, y)
        r = np.hypot(x, y)
        np.testing.assert_allclose(np.hypot(ax, ay), 1.3 ** (gamma - 1) * r ** (2 - gamma), rtol=1e-13)


def _epl_schramm(xv, yv, theta_e, gamma, q, phi):
    """Deflection of an elliptical convergence by the Schramm (1990) / Keeton (2001) 1-D
    integrals: with xi^2 = x'^2 + y'^2/q^2 and kappa(xi) = (3-gamma)/2 (theta_E/(sqrt(q) xi))^(gamma-1),
    a'_x = q x' J0, a'_y = q y' J1, J_n = int_0^1 kappa(xi(u)) / (1 - (1-q^2) u)^(n+1/2) du,
    xi(u)^2 = u (x'^2 + y'^2 / (1 - (1-q^2) u))."""
    xp, yp = _ell_frame(xv, yv, phi, 0.0, 0.0)
    e = gamma - 1.0
    C = (3.0 - gamma) / 2.0 * (theta_e / math.sqrt(q)) ** e

    def J(n):
        f = lambda u: C * (xp * xp + yp * yp / (1 - (1 - q * q) * u)) ** (-e / 2) / (1 - (1 - q * q) * u) ** (n + 0.5)
        val, _ = integrate.quad(f, 0.0, 1.0, weight="alg", wvar=(-e / 2, 0.0), epsabs=0, epsrel=1e-13, limit=200)
        return val

    apx, apy = q * xp * J(0), q * yp * J(1)
    return math.cos(phi) * apx - math.sin(phi) * apy, math.sin(phi) * apx + math.cos(phi) * apy


@pytest.mark.parametrize("gamma,q,phi", [(1.8, 0.6, 0.4), (2.2, 0.75, 2.0), (2.0, 0.5, 0.0), (1.9, 0.92, 1.1)])
def test_epl_matches_schramm_quadrature(gamma, q, phi):
    pts = [(0.7, 0.2), (-1.3, 0.9), (0.05, -1.8), (2.5, -2.1), (-0.3, -0.01)]
    for xv, yv in pts:
        ex, ey = _epl_schramm(xv, yv, 1.15, gamma, q, phi)
        ax, ay = oracle.alpha("EPL", [1.15, gamma, q, phi, 0.0, 0.0], [xv], [yv])
        assert abs(ax[0] - ex) < 1e-10 * max(1.0, abs(ex)), (xv, yv, ax[0], ex)
        assert abs(ay[0] - ey) < 1e-10 * max(1.0, abs(ey)), (xv, yv, ay[0], ey)


def test_e1e2_parametrisation_matches_q_phi():
    q, phi = 0.7, 0.6
    c = (1 - q) / (1 + q)
    e1, e2 = c * math.cos(2 * phi), c * math.sin(2 * phi)
    x, y = _pts(100, 9)
    a = oracle.alpha("EPL_E1E2", [1.0, 2.1, e1, e2, 0.1, 0.0], x, y)
    b = oracle.alpha("EPL", [1.0, 2.1, q, phi, 0.1, 0.0], x, y)
    np.testing.assert_allclose(a[0], b[0], rtol=1e-12, atol=1e-14)
    i1 = oracle.light("SERSIC_ELLIPSE", [3.0, 0.2, 2.0, e1, e2, 0.0, 0.1], x, y)
    i2 = oracle.light("SERSIC_ELLIPSE_Q_PHI", [3.0, 0.2, 2.0, q, phi, 0.0, 0.1], x, y)
    np.testing.assert_allclose(i1, i2, rtol=1e-12)


# ----------------------------------------------------------------------------- NFW / TNFW
def _rho(r, tau=None):
    base = 1.0 / (r * (1.0 + r) ** 2)
    return base if tau is None else base * tau * tau / (tau * tau + r * r)


def _m_quad(x, tau=None):
    """Dimensionless projected mass inside radius x: m(x) = (1/2) int_0^x x' Sigma(x') dx'
    = int_0^inf r^2 rho(r) g(r, x) dr, g = 1 inside the cylinder's sphere and
    1 - sqrt(1 - x^2/r^2) outside (the fraction of a shell inside the cylinder)."""
    inner, _ = integrate.quad(lambda r: r * r * _rho(r, tau), 0.0, x, epsabs=0, epsrel=1e-13, limit=400)
    g = lambda r: r * r * _rho(r, tau) * (x * x / (r * r)) / (1.0 + math.sqrt(1.0 - x * x / (r * r)))
    outer, _ = integrate.quad(g, x, np.inf, epsabs=0, epsrel=1e-13, limit=400)
    return inner + outer


def _sigma_quad(x, tau=None):
    """Projected dimensionless density Sigma(x) = 2 int_0^inf rho(sqrt(x^2+z^2)) dz."""
    v, _ = integrate.quad(lambda z: _rho(math.sqrt(x * x + z * z), tau), 0.0, np.inf, epsabs=0,
                          epsrel=1e-12, limit=400)
    return 2.0 * v


def _oracle_M(name, xs, Rs=0.02, ars=3e-3, rt=None):
    """Recover M(x) from the oracle's deflection magnitude along a ray at angle 0.7 rad."""
    out = []
    for xx in xs:
        r = xx * Rs
        px, py = 0.1 + r * math.cos(0.7), -0.2 + r * math.sin(0.7)
        p = [Rs, ars, 0.1, -0.2] if name == "NFW" else [Rs, ars, rt, 0.1, -0.2]
        ax, ay = oracle.alpha(name, p, [px], [py])
        out.append(math.hypot(ax[0], ay[0]) * xx * (1 - LN2) / ars)
    return np.array(out)


XS = [1e-3, 0.1, 0.5, 0.999, 1.0, 1.001, 2.0, 10.0, 100.0, 1e3]


def test_nfw_alpha_rs_normalisation():
    # alpha(Rs) = alpha_Rs, and the mass inside Rs is 1 - ln 2 by quadrature
    assert abs(_m_quad(1.0) - (1 - LN2)) < 1e-12
    M = _oracle_M("NFW", [1.0])
    assert abs(M[0] - (1 - LN2)) < 1e-12


def test_nfw_enclosed_mass_matches_density_quadrature():
    M = _oracle_M("NFW", XS)
    ref = np.array([_m_quad(x) for x in XS])
    np.testing.assert_allclose(M, ref, rtol=1e-9)


@pytest.mark.parametrize("tau", [5.0, 2.0, 20.0])
def test_tnfw_enclosed_mass_matches_density_quadrature(tau):
    Rs = 0.02
    M = _oracle_M("TNFW", XS, Rs=Rs, rt=tau * Rs)
    ref = np.array([_m_quad(x, tau) for x in XS])
    np.testing.assert_allclose(M, ref, rtol=1e-9)


def test_tnfw_limits():
    Rs = 0.03
    xs = [0.05, 0.7, 3.0, 12.0]
    # tau -> infinity recovers NFW (truncation correction ~ x^2 ln / tau^2)
    big = _oracle_M("TNFW", xs, Rs=Rs, rt=1e5 * Rs)
    nfw = _oracle_M("NFW", xs, Rs=Rs)
    np.testing.assert_allclose(big, nfw, rtol=1e-7)
    # r -> infinity: point mass of the total mass (total from the density quadrature)
    tau = 5.0
    mtot, _ = integrate.quad(lambda r: r * r * _rho(r, tau), 0, np.inf, epsabs=0, epsrel=1e-13, limit=400)
    far = _oracle_M("TNFW", [1e6], Rs=Rs, rt=tau * Rs)
    assert abs(far[0] - mtot) < 1e-5 * mtot


@pytest.mark.parametrize("name,tau", [("NFW", None), ("TNFW", 5.0)])
def test_nfw_tnfw_divergence_is_twice_kappa(name, tau):
    Rs, ars = 0.05, 4e-3
    ks = ars / (4 * (1 - LN2) * Rs)
    p = [Rs, ars, 0.0, 0.0] if name == "NFW" else [Rs, ars, tau * Rs, 0.0, 0.0]
    for xx in (0.3, 0.9, 1.7, 6.0):
        px, py = np.array([xx * Rs * math.cos(1.1)]), np.array([xx * Rs * math.sin(1.1)])
        div, curl = _fd_div_curl(name, p, px, py, 1e-5 * Rs)
        kap = ks * _sigma_quad(xx, tau)
        assert abs(div[0] - 2 * kap) < 1e-6 * 2 * kap, (xx, div[0], 2 * kap)
        assert abs(curl[0]) < 1e-6 * 2 * kap


# ----------------------------------------------------------------------------- Sersic
def _sersic_flux(amp, Rs, n):
    bn = 1.9992 * n - 0.3271
    return 2 * math.pi * n * Rs * Rs * amp * math.exp(bn) * bn ** (-2 * n) * special.gamma(2 * n)


@pytest.mark.parametrize("n", [0.5, 1.0, 2.5, 4.0])
def test_sersic_total_flux_radial_quadrature(n):
    amp, Rs, q, phi = 7.0, 0.3, 0.65, 0.8
    # along the major axis x', R = sqrt(q) x'
    def I_of_R(R):
        xp = R / math.sqrt(q)
        return oracle.light("SERSIC_ELLIPSE_Q_PHI", [amp, Rs, n, q, phi, 0.0, 0.0],
                            [xp * math.cos(phi)], [xp * math.sin(phi)])[0]
    tot, _ = integrate.quad(lambda R: 2 * math.pi * R * I_of_R(R), 0, np.inf, epsabs=0, epsrel=1e-11,
                            limit=500, points=None)
    assert abs(tot - _sersic_flux(amp, Rs, n)) < 1e-8 * tot


def test_unlensed_image_sums_to_sersic_flux():
    # no deflector: the image is the source binned on the grid; flux per pixel sums to the total
    sysm = W.LensSystem(W.Grid(300, 300, 5, 0.04), [], np.zeros((5, 0), np.float32),
                        ("SERSIC_ELLIPSE_Q_PHI", [4.0, 0.3, 1.0, 0.6, 0.5, 0.1, -0.05]), None)
    img = oracle.image(sysm)
    assert abs(img.sum() - _sersic_flux(4.0, 0.3, 1.0)) < 1e-4 * img.sum()


def test_grid_orientation_and_centre():
    # source at (0.3, -0.2): brightest pixel at column 20 + 6, row 20 - 4 (+x right, rows = +y)
    sysm = W.LensSystem(W.Grid(41, 41, 1, 0.05), [], np.zeros((5, 0), np.float32),
                        ("SERSIC", [1.0, 0.1, 1.0, 0.3, -0.2]), None)
    img = oracle.image(sysm)
    i, j = np.unravel_index(np.argmax(img), img.shape)
    assert (i, j) == (16, 26)
    sysm.grid = W.Grid(41, 41, 1, 0.05, x0=0.3, y0=-0.2)
    img = oracle.image(sysm)
    assert np.unravel_index(np.argmax(img), img.shape) == (20, 20)


def test_supersampled_pixel_converges_to_pixel_integral():
    # midpoint-rule convergence O((dpix/s)^2) fixes the sub-pixel offsets
    src = ("SERSIC_ELLIPSE_Q_PHI", [2.0, 0.15, 1.0, 0.8, 0.2, 0.02, 0.01])
    d = 0.05
    exact, _ = integrate.dblquad(lambda yy, xx: oracle.light(src[0], src[1], [xx], [yy])[0],
                                 0.1 - d / 2, 0.1 + d / 2, 0.05 - d / 2, 0.05 + d / 2, epsabs=0, epsrel=1e-11)
    errs = []
    for s in (2, 4, 8):
        sysm = W.LensSystem(W.Grid(1, 1, s, d, x0=0.1, y0=0.05), [], np.zeros((5, 0), np.float32), src, None)
        errs.append(abs(oracle.image(sysm)[0, 0] - exact))
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


# ----------------------------------------------------------------------------- PSF convolution
def test_delta_psf_is_identity():
    img = np.random.default_rng(10).random((17, 23))
    K = np.zeros((5, 5)); K[2, 2] = 1.0
    np.testing.assert_array_equal(oracle.convolve(img, K), img)


@pytest.mark.parametrize("k", [1, 3, 5, 13, 21])
def test_convolution_matches_scipy(k):
    rng = np.random.default_rng(k)
    img = rng.random((40, 37))
    K = rng.random((k, k))  # asymmetric on purpose: fixes the flip convention
    ref = signal.convolve2d(img, K, mode="same", boundary="fill")
    np.testing.assert_allclose(oracle.convolve(img, K), ref, rtol=1e-12, atol=1e-12)
    ref2 = signal.fftconvolve(img, K, mode="same")
    np.testing.assert_allclose(oracle.convolve(img, K), ref2, rtol=1e-9, atol=1e-9)


def test_normalised_psf_conserves_flux_and_adjoint():
    rng = np.random.default_rng(11)
    img = np.zeros((50, 50)); img[12:38, 10:40] = rng.random((26, 30))
    K = W.moffat_psf(3.0, 0.12, 0.04, 21).astype(np.float64)
    K /= K.sum()
    out = oracle.convolve(img, K)
    assert abs(out.sum() - img.sum()) < 1e-12 * img.sum()
    # dot-product test: <K x, y> = <x, K^T y>
    x = rng.standard_normal((31, 29)); y = rng.standard_normal((31, 29))
    Kr = rng.random((7, 7))
    lhs = np.sum(oracle.convolve(x, Kr) * y)
    rhs = np.sum(x * oracle.correlate(y, Kr))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


# ----------------------------------------------------------------------------- likelihood
def _small_diff(seed=3):
    return W.diff_problem(seed, n_points=4, n_sub=20, nx=24, dpix=0.1, k=5)


def test_loglike_maximum_at_noise_free_truth():
    pb = _small_diff()
    model = oracle.model_image(pb.system, pb.truth)
    L, G = oracle.loglike(pb.system, model, 0.01, 1000.0, pb.truth[None, :])
    assert abs(L[0]) < 1e-20
    assert np.abs(G).max() < 1e-10


def test_loglike_gradient_matches_central_differences():
    # central differences are O(h^2); Richardson extrapolation of h and h/2 makes them O(h^4)
    pb = _small_diff()
    data = W.observe(oracle.model_image(pb.system, pb.truth), 0.01, 1000.0, 5)
    P = pb.points.astype(np.float64)
    L, G = oracle.loglike(pb.system, data, 0.01, 1000.0, P)

    def cd(i, k, h):
        Pp = P[i].copy(); Pp[k] += h
        Pm = P[i].copy(); Pm[k] -= h
        return (oracle.loglike(pb.system, data, 0.01, 1000.0, Pp[None], grad=False)[0]
                - oracle.loglike(pb.system, data, 0.01, 1000.0, Pm[None], grad=False)[0]) / (2 * h)

    for i in range(2):
        for k in range(15):
            h = 1e-4 * max(1.0, abs(P[i, k]))
            d1 = cd(i, k, h)
            rich = (4 * cd(i, k, h / 2) - d1) / 3
            scale = max(abs(G[i, k]), 1e-3 * np.abs(G[i]).max())
            assert abs(rich - G[i, k]) < 1e-7 * scale, (i, k, rich, G[i, k])


def test_loglike_reduces_to_gaussian_chi2_without_poisson_term():
    pb = _small_diff()
    m = oracle.model_image(pb.system, pb.points[0])
    data = W.observe(m, 0.01, 1000.0, 7)
    L = oracle.loglike(pb.system, data, 0.02, 1e30, pb.points[:1], grad=False)
    chi2 = np.sum((data.astype(np.float64) - m) ** 2) / 0.02 ** 2
    assert abs(L[0] + 0.5 * chi2) < 1e-9 * chi2


def test_loglike_variance_model_matches_the_noise_law():
    # Pins the pixel variance of the likelihood, sigma^2 = sigma_bkg^2 + max(m, 0)/t_exp, against
    # the noise law itself: the observation generator draws Gaussian background noise of
    # variance sigma_bkg^2 plus Poisson counts of mean max(m, 0) t_exp divided by t_exp, whose
    # variance is max(m, 0)/t_exp.  Over many seeded draws at the truth, the oracle's
    # (d - m)^2 / sigma^2 must then average 1 per pixel, separately in pixels dominated by the
    # background and in pixels dominated by the Poisson term.  Each pixel group is isolated by
    # setting the data of every other pixel to the model (zero residual there).
    pb = _small_diff()
    sb, t = 0.01, 100.0
    m = oracle.model_image(pb.system, pb.truth)
    mp = np.maximum(m, 0.0)
    groups = {"background": mp / t <= 0.1 * sb ** 2, "poisson": mp / t >= 10.0 * sb ** 2}
    assert all(g.sum() >= 30 for g in groups.values()), {k: int(g.sum()) for k, g in groups.items()}
    n_seeds = 300
    chi = {k: [] for k in groups}
    alt = {("background", "data in place of the model"): [], ("poisson", "t_exp^2 in place of t_exp"): []}
    for seed in range(n_seeds):
        d = W.observe(m, sb, t, 5000 + seed).astype(np.float64)
        for name, mask in groups.items():
            dm = np.where(mask, d, m)
            L = oracle.loglike(pb.system, dm, sb, t, pb.truth[None, :], grad=False)[0]
            chi[name].append(-2.0 * L / mask.sum())
        r2 = (d - m) ** 2
        g = groups["background"]
        alt[("background", "data in place of the model")].append(
            np.mean(r2[g] / (sb ** 2 + np.maximum(d[g], 0.0) / t)))
        g = groups["poisson"]
        alt[("poisson", "t_exp^2 in place of t_exp")].append(np.mean(r2[g] / (sb ** 2 + mp[g] / t ** 2)))
    for name, v in chi.items():
        v = np.array(v)
        se = v.std(ddof=1) / math.sqrt(n_seeds)
        assert se < 0.03, (name, se)
        assert abs(v.mean() - 1.0) < 5.0 * se, (name, v.mean(), se)
    # the statistic separates the plausible misreadings of the variance by far more than its
    # sampling error (computed here from the same draws, outside the oracle)
    for (name, what), v in alt.items():
        v = np.array(v)
        se = np.array(chi[name]).std(ddof=1) / math.sqrt(n_seeds)
        assert abs(v.mean() - 1.0) > 20.0 * se, (name, what, v.mean(), se)


def test_conditioning_floor_mode_is_close_to_fp64():
    sysm = W.substructure_system(1, n_sub=200, nx=24, s=2, k=5)
    a = oracle.image(sysm)
    b = oracle.image(sysm, fp32=True)
    err = np.abs(a - b).max() / np.abs(a).max()
    assert 0 < err < 1e-4


def test_nfw_tnfw_mass_against_40_digit_golden():
    """tests/golden/nfw_tnfw_mass.txt: mpmath quadrature of the 3-D densities (make_golden.py)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "nfw_tnfw_mass.txt")
    rows = [l.split() for l in open(path) if not l.startswith("#")]
    xs = [float(r[0]) for r in rows]
    nfw = np.array([float(r[1]) for r in rows])
    tnfw = np.array([float(r[2]) for r in rows])
    Rs = 0.02
    # atol: the plain FP64 formulas cancel terms of size ~ tau^2 ln(2/x) at small x
    np.testing.assert_allclose(_oracle_M("NFW", xs, Rs=Rs), nfw, rtol=2e-9, atol=1e-14)
    np.testing.assert_allclose(_oracle_M("TNFW", xs, Rs=Rs, rt=5 * Rs), tnfw, rtol=2e-9, atol=1e-14)


def test_linear_amplitude_recovers_truth_and_minimises_chi2():
    pb = _small_diff()
    truth = pb.truth.astype(np.float64)
    data = oracle.model_image(pb.system, truth)  # noise-free, amplitude truth[8]
    a, L = oracle.linear_amp(pb.system, data, 0.01, 1000.0, truth[None])
    assert abs(a[0] - truth[8]) < 1e-10 * truth[8] and abs(L[0]) < 1e-12
    # with noise the solution is the minimum of the weighted chi^2 along the amplitude
    noisy = W.observe(data, 0.01, 1000.0, 9).astype(np.float64)
    p = pb.points[0].astype(np.float64)
    a, L = oracle.linear_amp(pb.system, noisy, 0.01, 1000.0, p[None])
    w = 1.0 / (0.01 ** 2 + np.maximum(noisy, 0) / 1000.0)
    q = p.copy(); q[8] = 1.0
    m1 = oracle.model_image(pb.system, q)
    chi = lambda amp: np.sum(w * (noisy - amp * m1) ** 2)
    assert chi(a[0]) < chi(a[0] * (1 + 1e-4)) and chi(a[0]) < chi(a[0] * (1 - 1e-4))
    assert abs(L[0] + 0.5 * chi(a[0])) < 1e-9 * chi(a[0])


# ----------------------------------------------------------------------------- multipoles
def _kappa_multipole(x, y, m, am, phim, cx, cy, rE):
    # convergence of the m-th circular multipole: r_E a_m cos(m (phi - phi_m)) / (2 r)
    dx, dy = x - cx, y - cy
    return rE * am * np.cos(m * (np.arctan2(dy, dx) - phim)) / (2.0 * np.hypot(dx, dy))


@pytest.mark.parametrize("m", [1, 2, 3, 4, 6])
def test_multipole_divergence_is_twice_kappa_and_curl_free(m):
    p = [m, 0.07, 0.4, 0.1, -0.15, 1.3]
    x, y = _pts(400, 40 + m, -2.5, 2.5)
    r = np.hypot(x - 0.1, y + 0.15)
    x, y = x[r > 0.2], y[r > 0.2]
    div, curl = _fd_div_curl("MULTIPOLE", p, x, y, 1e-5)
    k = _kappa_multipole(x, y, *p)
    scale = np.abs(2 * k).max()
    assert np.abs(div - 2 * k).max() < 1e-7 * scale
    assert np.abs(curl).max() < 1e-7 * scale


def _multipole_potential(x, y, m, am, phim, cx, cy, rE):
    dx, dy = x - cx, y - cy
    r = np.hypot(dx, dy)
    d = np.arctan2(dy, dx) - phim
    if m == 1:
        return 0.5 * rE * am * r * np.log(r / rE) * np.cos(d)
    return rE * am * r * np.cos(m * d) / (1.0 - m * m)


@pytest.mark.parametrize("m", [1, 2, 4])
def test_multipole_deflection_is_gradient_of_its_potential(m):
    # the defining potential, differentiated numerically (Richardson-extrapolated central
    # differences), against the oracle's analytic radial/tangential derivatives
    p = [m, 0.05, -0.7, 0.0, 0.2, 0.9]
    x, y = _pts(200, 50 + m, -2.0, 2.0)
    x, y = x[np.hypot(x, y - 0.2) > 0.3], y[np.hypot(x, y - 0.2) > 0.3]

    def grad(h):
        gx = (_multipole_potential(x + h, y, *p) - _multipole_potential(x - h, y, *p)) / (2 * h)
        gy = (_multipole_potential(x, y + h, *p) - _multipole_potential(x, y - h, *p)) / (2 * h)
        return gx, gy
    g1, g2 = grad(1e-3), grad(5e-4)
    gx = (4 * g2[0] - g1[0]) / 3
    gy = (4 * g2[1] - g1[1]) / 3
    ax, ay = oracle.alpha("MULTIPOLE", p, x, y)
    scale = np.abs(np.concatenate([ax, ay])).max()
    assert np.abs(ax - gx).max() < 1e-9 * scale and np.abs(ay - gy).max() < 1e-9 * scale


def test_multipole_m_ge_2_is_scale_free_and_rotates_with_phi_m():
    # alpha of an m >= 2 multipole is homogeneous of degree 0 in r; turning phi_m by t turns
    # the pattern by t
    p = [3, 0.04, 0.3, 0.0, 0.0, 1.1]
    x, y = _pts(100, 61, -1.5, 1.5)
    a1 = oracle.alpha("MULTIPOLE", p, x, y)
    a2 = oracle.alpha("MULTIPOLE", p, 2.7 * x, 2.7 * y)
    np.testing.assert_allclose(a2[0], a1[0], rtol=0, atol=1e-15)
    np.testing.assert_allclose(a2[1], a1[1], rtol=0, atol=1e-15)
    t = 0.45
    c, s = math.cos(t), math.sin(t)
    q = list(p); q[2] = p[2] + t
    b = oracle.alpha("MULTIPOLE", q, c * x - s * y, s * x + c * y)
    np.testing.assert_allclose(b[0], c * a1[0] - s * a1[1], atol=1e-14)
    np.testing.assert_allclose(b[1], s * a1[0] + c * a1[1], atol=1e-14)


def test_epl_multipole_m1m3m4_is_epl_plus_three_multipoles():
    th, g, e1, e2, cx, cy = 1.1, 2.05, 0.05, -0.03, 0.01, 0.02
    a = [(1, 0.01, 0.2), (3, 0.02, 0.1), (4, 0.015, -0.3)]
    p = [th, g, e1, e2, cx, cy] + [v for _, am, dp in a for v in (am, dp)]
    x, y = _pts(300, 62)
    ax, ay = oracle.alpha("EPL_MULTIPOLE_M1M3M4", p, x, y)
    rx, ry = oracle.alpha("EPL_E1E2", [th, g, e1, e2, cx, cy], x, y)
    phi = 0.5 * math.atan2(e2, e1)
    for m, am, dp in a:
        mx, my = oracle.alpha("MULTIPOLE", [m, am, phi + dp, cx, cy, th], x, y)
        rx, ry = rx + mx, ry + my
    np.testing.assert_allclose(ax, rx, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(ay, ry, rtol=1e-13, atol=1e-15)
    # zero amplitudes reduce it to the EPL exactly
    z = [th, g, e1, e2, cx, cy, 0.0, 0.3, 0.0, 1.0, 0.0, -2.0]
    np.testing.assert_array_equal(oracle.alpha("EPL_MULTIPOLE_M1M3M4", z, x, y)[0],
                                  oracle.alpha("EPL_E1E2", z[:6], x, y)[0])


# ----------------------------------------------------------------------------- shapelets
def _shapelet_index(nmax):
    return [(n1, n - n1) for n in range(nmax + 1) for n1 in range(n, -1, -1)]


def _phi_numpy(n, u):
    # physicists' Hermite polynomial from numpy's library routine, with the orthonormal weight
    from numpy.polynomial import hermite
    c = np.zeros(n + 1); c[n] = 1.0
    return hermite.hermval(u, c) * np.exp(-0.5 * u * u) / math.sqrt(2.0 ** n * math.factorial(n) * math.sqrt(math.pi))


def test_shapelet_basis_matches_numpy_hermite():
    nmax, beta, cx, cy = 8, 0.35, 0.05, -0.1
    x, y = _pts(300, 70, -1.5, 1.5)
    idx = _shapelet_index(nmax)
    for k in (0, 1, 2, 5, 11, 20, 44):
        c = np.zeros(len(idx)); c[k] = 1.0
        n1, n2 = idx[k]
        got = oracle.light("SHAPELETS", [nmax, beta, cx, cy], x, y, coeffs=c)
        ref = _phi_numpy(n1, (x - cx) / beta) * _phi_numpy(n2, (y - cy) / beta) / beta
        np.testing.assert_allclose(got, ref, rtol=1e-11, atol=1e-13)


def test_shapelet_basis_is_orthonormal_and_ordered():
    # Gram matrix by the trapezoid rule on a wide fine grid (spectrally accurate for these
    # Gaussian-damped functions), and parity of each basis function: B_(n1,n2) has parity
    # (-1)^n1 in x and (-1)^n2 in y, which fixes the amplitude ordering
    nmax, beta = 4, 0.5
    idx = _shapelet_index(nmax)
    g = np.linspace(-6.0, 6.0, 481)
    X, Y = np.meshgrid(g, g)
    dA = (g[1] - g[0]) ** 2
    B = []
    for k in range(len(idx)):
        c = np.zeros(len(idx)); c[k] = 1.0
        B.append(oracle.light("SHAPELETS", [nmax, beta, 0.0, 0.0], X.ravel(), Y.ravel(), coeffs=c))
    B = np.array(B)
    gram = B @ B.T * dA
    np.testing.assert_allclose(gram, np.eye(len(idx)), atol=1e-10)
    x, y = _pts(50, 71, 0.1, 1.0)
    for k, (n1, n2) in enumerate(idx):
        c = np.zeros(len(idx)); c[k] = 1.0
        f = lambda u, v: oracle.light("SHAPELETS", [nmax, beta, 0.0, 0.0], u, v, coeffs=c)
        np.testing.assert_allclose(f(-x, y), (-1) ** n1 * f(x, y), atol=1e-14)
        np.testing.assert_allclose(f(x, -y), (-1) ** n2 * f(x, y), atol=1e-14)


def _shapelet_flux(nmax, beta, coeffs):
    # closed form: int phi_n du = pi^(1/4) 2^((1-n)/2) sqrt(n!) / (n/2)! for even n, 0 for odd n
    def f1(n):
        if n % 2:
            return 0.0
        return math.pi ** 0.25 * 2.0 ** ((1 - n) / 2) * math.sqrt(math.factorial(n)) / math.factorial(n // 2)
    return sum(c * f1(n1) * f1(n2) * beta for c, (n1, n2) in zip(coeffs, _shapelet_index(nmax)))


def test_unlensed_shapelet_image_sums_to_closed_form_flux():
    nmax, beta = 6, 0.3
    coeffs = np.random.default_rng(72).normal(size=(nmax + 1) * (nmax + 2) // 2)
    system = W.LensSystem(W.Grid(120, 120, 2, 0.05), [], np.zeros((5, 0), np.float32),
                          ("SHAPELETS", [nmax, beta, 0.02, -0.03]), None, coeffs)
    img = oracle.image(system)
    flux = _shapelet_flux(nmax, beta, coeffs)
    assert abs(img.sum() - flux) < 1e-8 * np.abs(coeffs).sum()


# ----------------------------------------------------------------------------- cored steep ellipsoid
def _kappa_cse(x, y, A, s, e1, e2, cx, cy):
    phi = 0.5 * math.atan2(e2, e1)
    c = math.hypot(e1, e2)
    q = (1 - c) / (1 + c)
    xp, yp = _ell_frame(x, y, phi, cx, cy)
    return A / (2.0 * (s * s + xp * xp + yp * yp / (q * q)) ** 1.5)


@pytest.mark.parametrize("p", [[0.5, 0.2, 0.2, -0.1, 0.1, 0.0], [1.3, 0.03, 0.35, 0.2, 0.0, 0.1],
                               [0.1, 1.5, -0.4, 0.1, 0.0, 0.0]])
def test_cse_divergence_is_twice_kappa_and_curl_free(p):
    x, y = _pts(300, 80)
    div, curl = _fd_div_curl("CSE", p, x, y, 1e-5)
    k = _kappa_cse(x, y, *p)
    np.testing.assert_allclose(div, 2 * k, rtol=2e-7, atol=1e-9 * np.abs(k).max())
    assert np.abs(curl).max() < 1e-7 * np.abs(2 * k).max()


def test_cse_round_closed_form():
    # q = 1: enclosed mass of A / (2 (s^2 + r^2)^(3/2)) gives alpha = (A/r)(1/s - 1/sqrt(s^2 + r^2))
    A, s = 0.7, 0.15
    x, y = _pts(300, 81, -4.0, 4.0)
    ax, ay = oracle.alpha("CSE", [A, s, 0.0, 0.0, 0.2, -0.1], x, y)
    r = np.hypot(x - 0.2, y + 0.1)
    np.testing.assert_allclose(np.hypot(ax, ay), (A / r) * (1 / s - 1 / np.sqrt(s * s + r * r)), rtol=1e-12)
    np.testing.assert_allclose(ax * (y + 0.1) - ay * (x - 0.2), 0.0, atol=1e-13)


# ----------------------------------------------------------------------------- elliptical NFW / Hernquist
def _F_scalar(x):
    if x < 1:
        return math.acosh(1 / x) / math.sqrt(1 - x * x)
    if x > 1:
        return math.acos(1 / x) / math.sqrt(x * x - 1)
    return 1.0


def _kappa_hat(name, x):
    # projected NFW (Bartelmann 1996) and Hernquist (Hernquist 1990) profiles, written from the
    # 3-D densities' standard projections; x = 1 by its limit
    v = x * x - 1
    if name == "NFW_ELLIPSE_CSE":
        return 2 / 3 if v == 0 else 2 * (1 - _F_scalar(x)) / v
    return 4 / 15 if v == 0 else ((2 + x * x) * _F_scalar(x) - 3) / (v * v)


def _kappa_ell(name, p, x, y):
    a, Rs = (p[1] / (4 * (1 - LN2) * p[0]), p[0]) if name == "NFW_ELLIPSE_CSE" else (p[0], p[1])
    phi = 0.5 * math.atan2(p[3], p[2])
    c = math.hypot(p[2], p[3])
    q = (1 - c) / (1 + c)
    xp, yp = _ell_frame(x, y, phi, p[4], p[5])
    xi = np.sqrt(q * xp * xp + yp * yp / q)
    return np.array([a * _kappa_hat(name, v / Rs) for v in xi])


def test_nfw_ellipse_round_equals_nfw_closed_form():
    x, y = _pts(300, 90, -3.0, 3.0)
    ax, ay = oracle.alpha("NFW_ELLIPSE_CSE", [0.8, 0.3, 0.0, 0.0, 0.05, -0.1], x, y)
    rx, ry = oracle.alpha("NFW", [0.8, 0.3, 0.05, -0.1], x, y)
    np.testing.assert_allclose(ax, rx, rtol=1e-11, atol=1e-14)
    np.testing.assert_allclose(ay, ry, rtol=1e-11, atol=1e-14)


@pytest.mark.parametrize("name,p", [("NFW_ELLIPSE_CSE", [0.8, 0.3, 0.15, -0.2, 0.05, 0.0]),
                                    ("NFW_ELLIPSE_CSE", [0.2, 0.05, -0.3, 0.1, 0.0, 0.0]),
                                    ("HERNQUIST_ELLIPSE_CSE", [0.5, 0.8, 0.1, -0.2, 0.0, 0.1]),
                                    ("HERNQUIST_ELLIPSE_CSE", [1.2, 0.3, 0.25, 0.2, 0.0, 0.0])])
def test_nfw_hernquist_ellipse_divergence_is_twice_kappa(name, p):
    x, y = _pts(150, 91, -2.5, 2.5)
    keep = np.hypot(x - p[4], y - p[5]) > 0.05
    x, y = x[keep], y[keep]
    div, curl = _fd_div_curl(name, p, x, y, 1e-5)
    k = _kappa_ell(name, p, x, y)
    np.testing.assert_allclose(div, 2 * k, rtol=1e-6, atol=1e-8 * np.abs(k).max())
    assert np.abs(curl).max() < 1e-6 * np.abs(2 * k).max()


def test_hernquist_round_enclosed_mass():
    # alpha(r) = (2/r) int_0^r kappa r' dr' by 60-digit quadrature of the projected profile (the
    # closed form cancels badly near x = 1 in FP64, so the reference runs in mpmath); and the
    # profile integrates to unit mass, int_0^inf kappa_hat x dx = 1
    mpmath = pytest.importorskip("mpmath")
    mp = mpmath.mp
    mp.dps = 60

    def kh(x):
        x = mp.mpf(x)
        if abs(x * x - 1) < mp.mpf(10) ** -20:   # the limit; the next term is 8/35 (x^2 - 1)
            return mp.mpf(4) / 15
        F = mp.acosh(1 / x) / mp.sqrt(1 - x * x) if x < 1 else mp.acos(1 / x) / mp.sqrt(x * x - 1)
        return ((2 + x * x) * F - 3) / (x * x - 1) ** 2

    sigma0, Rs = 0.6, 0.4
    r = np.array([0.01, 0.1, 0.39, 0.4, 0.41, 1.0, 3.0, 10.0])
    ax, ay = oracle.alpha("HERNQUIST_ELLIPSE_CSE", [sigma0, Rs, 0.0, 0.0, 0.0, 0.0], r, np.zeros_like(r))
    ref = []
    for v in r:
        pts = [0, min(v, Rs), v] if v > Rs else [0, v]
        ref.append(float(2 * sigma0 * mp.quad(lambda t: kh(t / Rs) * t, pts) / v))
    np.testing.assert_allclose(ax, ref, rtol=1e-11)
    assert np.abs(ay).max() < 1e-15
    assert abs(mp.quad(lambda t: kh(t) * t, [0, 1, 10, mp.inf]) - 1) < 1e-12


# ----------------------------------------------------------------------------- elliptical multipoles
def _kappa_multipole_ell(x, y, m, am, phim, q, phie, cx, cy, rE):
    # reading: r_E a_m cos(m (varphi - (phi_m - phi_e))) / (2 R) in the ellipse frame,
    # R^2 = q x''^2 + y''^2 / q, varphi = atan2(y'' / sqrt(q), x'' sqrt(q))
    dx, dy = x - cx, y - cy
    xp = math.cos(phie) * dx + math.sin(phie) * dy
    yp = -math.sin(phie) * dx + math.cos(phie) * dy
    R = np.sqrt(q * xp * xp + yp * yp / q)
    vphi = np.arctan2(yp / math.sqrt(q), xp * math.sqrt(q))
    return rE * am * np.cos(m * (vphi - (phim - phie))) / (2.0 * R)


@pytest.mark.parametrize("m", [1, 2, 3, 4, 6])
def test_elliptical_multipole_round_limit_is_the_circular_multipole(m):
    # q = 1: the ellipse orientation drops out and the mode is the circular multipole, whose
    # oracle (complex powers of the direction) is pinned above
    x, y = _pts(300, 70 + m, -2.0, 2.0)
    circ = oracle.alpha("MULTIPOLE", [m, 0.06, 0.35, 0.1, -0.2, 1.2], x, y)
    ell = oracle.alpha("MULTIPOLE_ELL", [m, 0.06, 0.35, 1.0, 0.9, 0.1, -0.2, 1.2], x, y)
    scale = np.abs(np.concatenate(circ)).max()
    assert np.abs(ell[0] - circ[0]).max() < 1e-12 * scale
    assert np.abs(ell[1] - circ[1]).max() < 1e-12 * scale


@pytest.mark.parametrize("m,q", [(1, 0.6), (2, 0.5), (3, 0.8), (4, 0.7), (4, 0.25), (7, 0.55)])
def test_elliptical_multipole_divergence_is_twice_kappa_and_curl_free(m, q):
    p = [m, 0.05, 0.7, q, -0.4, 0.05, 0.1, 1.1]
    x, y = _pts(300, 80 + m, -2.5, 2.5)
    keep = np.hypot(x - 0.05, y - 0.1) > 0.2
    x, y = x[keep], y[keep]
    div, curl = _fd_div_curl("MULTIPOLE_ELL", p, x, y, 1e-5)
    k = _kappa_multipole_ell(x, y, *p)
    scale = np.abs(2 * k).max()
    assert np.abs(div - 2 * k).max() < 1e-7 * scale
    assert np.abs(curl).max() < 1e-7 * scale


def test_elliptical_multipole_rotates_with_its_angles():
    # turning the ellipse and the multipole phase by t turns the deflection field by t
    p = [3, 0.04, 0.3, 0.6, 1.1, 0.0, 0.0, 1.0]
    x, y = _pts(100, 91, -1.5, 1.5)
    a = oracle.alpha("MULTIPOLE_ELL", p, x, y)
    t = 0.7
    c, s = math.cos(t), math.sin(t)
    q = list(p); q[2] += t; q[4] += t
    b = oracle.alpha("MULTIPOLE_ELL", q, c * x - s * y, s * x + c * y)
    np.testing.assert_allclose(b[0], c * a[0] - s * a[1], atol=1e-13)
    np.testing.assert_allclose(b[1], s * a[0] + c * a[1], atol=1e-13)


@pytest.mark.parametrize("m", [2, 4])
def test_elliptical_multipole_even_orders_are_scale_free(m):
    # for even m, 2 kappa r is unchanged under theta -> theta + pi, so it has no k = +-1
    # harmonic: the potential is r F(theta) and alpha is homogeneous of degree 0 in r
    p = [m, 0.05, 0.2, 0.55, 0.3, 0.0, 0.0, 1.3]
    x, y = _pts(100, 95 + m, -1.5, 1.5)
    a1 = oracle.alpha("MULTIPOLE_ELL", p, x, y)
    a2 = oracle.alpha("MULTIPOLE_ELL", p, 3.1 * x, 3.1 * y)
    np.testing.assert_allclose(a2[0], a1[0], rtol=0, atol=1e-14)
    np.testing.assert_allclose(a2[1], a1[1], rtol=0, atol=1e-14)


def test_elliptical_multipole_rejects_out_of_range_parameters():
    x, y = _pts(4, 3)
    for bad in ([0, 0.05, 0.0, 0.6, 0.0, 0.0, 0.0, 1.0], [2.5, 0.05, 0.0, 0.6, 0.0, 0.0, 0.0, 1.0],
                [2, 0.05, 0.0, 0.1, 0.0, 0.0, 0.0, 1.0], [2, 0.05, 0.0, 0.6, 0.0, 0.0, 0.0, 0.0]):
        with pytest.raises(ValueError):
            oracle.alpha("MULTIPOLE_ELL", bad, x, y)

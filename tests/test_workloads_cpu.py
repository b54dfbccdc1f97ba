"""The seeded input generators follow the stated recipe of each workload (the shapes, ranges and
distributions of the paper's workloads; no dataset): determinism, the subhalo population's
distributions, PSF normalisation, parameter ranges, the batched and serving mixes, and the
observation noise model."""
import math

import numpy as np
import pytest

from paper_2606_01547_gb300 import workloads as W

scipy_stats = pytest.importorskip("scipy.stats")


def test_same_seed_same_inputs_and_seeds_differ():
    a, b, c = W.substructure_system(5), W.substructure_system(5), W.substructure_system(6)
    np.testing.assert_array_equal(a.subhalos, b.subhalos)
    assert a.deflectors == b.deflectors and a.source == b.source
    assert not np.array_equal(a.subhalos, c.subhalos)
    assert a.deflectors != c.deflectors


def test_subhalo_population_distributions():
    sub = W.subhalo_population(W._rng(11), 20000).astype(np.float64)
    assert sub.shape == (5, 20000) and sub.dtype == np.float64
    cx, cy, rs, ars, rt = sub
    r2 = cx * cx + cy * cy
    assert r2.max() <= 9.0 * (1 + 1e-6)
    # uniform in the 3" disc: r^2 / 9 ~ U[0, 1], the angle ~ U[0, 2 pi)
    assert scipy_stats.kstest(r2 / 9.0, "uniform").pvalue > 1e-3
    assert scipy_stats.kstest((np.arctan2(cy, cx) + np.pi) / (2 * np.pi), "uniform").pvalue > 1e-3
    # Rs log-uniform in [0.005, 0.05]", alpha_Rs log-uniform in [1e-4, 1e-2]"
    for v, lo, hi in ((rs, 0.005, 0.05), (ars, 1e-4, 1e-2)):
        assert v.min() >= lo * (1 - 1e-6) and v.max() <= hi * (1 + 1e-6)
        u = (np.log(v) - math.log(lo)) / (math.log(hi) - math.log(lo))
        assert scipy_stats.kstest(np.clip(u, 0, 1), "uniform").pvalue > 1e-3
    # truncation r_t = 5 Rs (up to the FP32 rounding of both)
    np.testing.assert_allclose(rt, 5.0 * rs, rtol=2e-7)


@pytest.mark.parametrize("make", [lambda: W.gaussian_psf(0.1, 0.05, 5), lambda: W.gaussian_psf(0.1, 0.05, 13),
                                  lambda: W.moffat_psf(3.0, 0.12, 0.04, 21), lambda: W.moffat_psf(3.0, 0.12, 0.04, 31)])
def test_psf_kernels_are_normalised_symmetric_and_peaked(make):
    K = make().astype(np.float64)
    k = K.shape[0]
    assert K.shape == (k, k) and k % 2 == 1
    assert abs(K.sum() - 1.0) < 1e-6
    np.testing.assert_array_equal(K, K.T)
    np.testing.assert_array_equal(K, K[::-1, ::-1])
    c = k // 2
    assert K[c, c] == K.max()
    assert np.all(np.diff(K[c, c:]) < 0)  # falls off monotonically from the centre


def test_moffat_and_gaussian_widths():
    # the sampled kernels' half-maximum radius (from the defining profile) is the stated FWHM / 2
    for fwhm, dpix, beta in ((0.12, 0.04, 3.0), (0.3, 0.05, 2.5)):
        a = fwhm / (2.0 * math.sqrt(2.0 ** (1.0 / beta) - 1.0))
        assert abs((1.0 + (fwhm / 2) ** 2 / a ** 2) ** (-beta) - 0.5) < 1e-12
        K = W.moffat_psf(beta, fwhm, dpix, 61).astype(np.float64)
        c = 30
        # the centre row follows (1 + r^2/a^2)^-beta up to the normalisation
        r = np.arange(0, 5) * dpix
        prof = (1.0 + r * r / (a * a)) ** (-beta)
        np.testing.assert_allclose(K[c, c:c + 5] / K[c, c], prof, rtol=1e-6)
    sigma_px = 0.1 / (2 * math.sqrt(2 * math.log(2))) / 0.05
    G = W.gaussian_psf(0.1, 0.05, 41).astype(np.float64)
    yy, xx = np.mgrid[0:41, 0:41] - 20
    # sampled at pixel centres, a sigma = 0.85 px Gaussian's second moment is sigma^2 to ~4e-5
    np.testing.assert_allclose((G * xx * xx).sum(), sigma_px ** 2, rtol=1e-4)


def _qe(e1, e2):
    c = math.hypot(e1, e2)
    return (1 - c) / (1 + c)


def test_substructure_workload_recipe():
    for seed in range(20):
        sysm = W.substructure_system(seed)
        g = sysm.grid
        assert (g.nx, g.ny, g.s) == (200, 200, 3) and g.dpix == W.f32(0.04)
        (n1, epl), (n2, shear) = sysm.deflectors
        assert (n1, n2) == ("EPL", "SHEAR")
        theta_e, gamma, q, phi = epl[:4]
        assert 0.8 <= theta_e <= 1.4 and 1.8 <= gamma <= 2.2 and 0.6 <= q <= 0.95 and 0 <= phi < math.pi
        assert math.hypot(*shear) <= 0.08 + 1e-7
        name, src = sysm.source
        assert name == "SERSIC_ELLIPSE_Q_PHI"
        amp, r, n, qs = src[:4]
        assert amp == 10.0 and 0.05 <= r <= 0.5 and 0.5 <= n <= 4.0 and 0.6 <= qs <= 0.95
        assert max(abs(src[5]), abs(src[6])) <= 0.1
        assert sysm.n_sub == 10000 and sysm.psf.shape == (21, 21)
        assert sysm.pairs() == 360000 * 10000


def test_batched_mix_recipe():
    systems = W.batched_systems(3, count=300, max_sub=2000)
    assert len(systems) == 300
    seen_n, seen_s, seen_k = set(), set(), set()
    for sysm in systems:
        g = sysm.grid
        assert g.nx == g.ny and g.nx in W.BATCH_GRIDS and g.s in W.BATCH_SUPERSAMPLE
        k = sysm.psf.shape[0]
        assert k in W.BATCH_PSF
        assert 0 <= sysm.n_sub <= 2000
        seen_n.add(g.nx), seen_s.add(g.s), seen_k.add(k)
    assert seen_n == set(W.BATCH_GRIDS) and seen_s == set(W.BATCH_SUPERSAMPLE) and len(seen_k) >= 12
    # the count is floor(exp(U[0, ln 20001])) - 1, so P(count <= m) = ln(m + 2) / ln 20001
    rng = W._rng(4)
    n = 20000
    counts = np.array([W.log_uniform_count(rng, 20000) for _ in range(n)])
    assert counts.min() >= 0 and counts.max() <= 20000
    for m in (0, 1, 9, 99, 999, 9999):
        p = math.log(m + 2.0) / math.log(20001.0)
        assert abs((counts <= m).mean() - p) < 5 * math.sqrt(p * (1 - p) / n), m


def test_differentiation_workload_recipe():
    pb = W.diff_problem(9, n_points=64)
    g = pb.system.grid
    assert (g.nx, g.ny, g.s) == (100, 100, 1) and g.dpix == W.f32(0.05)
    assert pb.system.psf.shape == (13, 13) and pb.system.n_sub == 1000
    assert (pb.sigma_bkg, pb.t_exp) == (0.01, 1000.0)
    assert pb.points.shape == (64, 15) and pb.truth.shape == (15,)
    for p in np.concatenate([pb.truth[None], pb.points]):
        assert 0.8 <= p[0] <= 1.4 and 1.8 <= p[1] <= 2.2
        assert 0.6 - 1e-6 <= _qe(p[2], p[3]) <= 0.95 + 1e-6
        assert math.hypot(p[6], p[7]) <= 0.08 + 1e-7
        assert 5.0 <= p[8] <= 15.0 and 0.05 <= p[9] <= 0.5 and 0.5 <= p[10] <= 4.0
        assert 0.6 - 1e-6 <= _qe(p[11], p[12]) <= 0.95 + 1e-6


def test_serving_stream_recipe():
    rate, duration = 2000.0, 2.0
    reqs = W.serving_stream(1, rate=rate, duration=duration, max_sub=500)
    t = np.array([r.t_arrival for r in reqs])
    assert np.all(np.diff(t) > 0) and t[-1] < duration
    n = len(reqs)
    assert abs(n - rate * duration) < 5 * math.sqrt(rate * duration)  # Poisson count
    # exponential gaps: KS against the rate
    assert scipy_stats.kstest(np.diff(t) * rate, "expon").pvalue > 1e-3
    kinds = np.array([r.kind for r in reqs])
    frac = (kinds == 0).mean()
    assert abs(frac - 0.7) < 5 * math.sqrt(0.21 / n)
    for r in reqs:
        g = r.system.grid
        assert g.nx == g.ny and g.nx % 2 == 0 and 64 <= g.nx <= 256 and g.s == 1
        assert r.system.psf.shape[0] in W.BATCH_PSF and r.system.n_sub <= 500


def test_observation_noise_model():
    # d = m + N(0, sigma^2) + Poisson(max(m,0) t)/t - max(m,0): mean m, variance sigma^2 + max(m,0)/t
    sigma, t_exp = 0.01, 1000.0
    for m0 in (0.0, 0.05, 0.4):
        m = np.full((400, 400), m0)
        d = W.observe(m, sigma, t_exp, seed=int(m0 * 100)).astype(np.float64)
        var = sigma ** 2 + m0 / t_exp
        n = m.size
        assert abs(d.mean() - m0) < 5 * math.sqrt(var / n)
        assert abs(d.var() / var - 1.0) < 5 * math.sqrt(2.0 / n) + 1e-3
    neg = W.observe(np.full((200, 200), -0.1), sigma, t_exp, seed=3).astype(np.float64)
    assert abs(neg.var() / sigma ** 2 - 1.0) < 0.05  # no Poisson term below zero

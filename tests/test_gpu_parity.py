"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on seeded inputs.

Image tolerance: max|gpu - oracle| / max|oracle| <= max(1e-5, 2 * floor), where floor is
the same relative error of the oracle's conditioning-floor mode (FP64 arithmetic with the
grid, every deflection term and the traced position rounded to FP32).  That floor is the
error any FP32 evaluation must make; it only exceeds 1e-5 where a steep Sersic cusp meets
FP32 rounding of the traced coordinates.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2606_01547_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sim():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_01547_gb300 import lenssim
    s = lenssim.Simulator(device=0)
    yield s
    s.close()


def rel_linf(got, ref):
    return float(np.abs(np.asarray(got, np.float64) - ref).max() / np.abs(ref).max())


def image_tol(system, ref):
    floor = rel_linf(oracle.image(system, fp32=True), ref)
    return max(1e-5, 2.0 * floor), floor


def gpu_image(sim, system, **kw):
    out = sim.image(system, **kw)[0]
    torch.cuda.synchronize()
    return out.cpu().numpy()


# ----------------------------------------------------------------------------- whole images
def test_plain_60x60_image_matches_oracle(sim):
    system = W.plain_system()
    ref = oracle.image(system)
    err = rel_linf(gpu_image(sim, system), ref)
    assert err <= 1e-5, err


@pytest.mark.parametrize("seed,nx,s,nsub,k", [(0, 36, 3, 300, 7), (1, 29, 2, 77, 5), (2, 20, 1, 513, 1),
                                              (3, 17, 4, 40, 3), (4, 11, 5, 130, 9)])
def test_substructure_small_images_match_oracle(sim, seed, nx, s, nsub, k):
    # several 8x4 tiles with ragged edges; s = 4, 5 exercise the multi-pass sample path
    system = W.substructure_system(seed, n_sub=nsub, nx=nx, s=s, k=k)
    ref = oracle.image(system)
    tol, floor = image_tol(system, ref)
    err = rel_linf(gpu_image(sim, system), ref)
    assert err <= tol, (err, floor)


@pytest.mark.parametrize("seed,n_max,nx,s,nsub,k", [(0, 6, 44, 2, 300, 5), (1, 10, 37, 3, 120, 7),
                                                     (2, 0, 25, 1, 0, 3), (3, 3, 30, 2, 50, 0)])
def test_multipole_lens_and_shapelet_source_images_match_oracle(sim, seed, n_max, nx, s, nsub, k):
    system = W.multipole_shapelet_system(seed, n_max=n_max, n_sub=nsub, nx=nx, s=s, k=k)
    ref = oracle.image(system)
    tol, floor = image_tol(system, ref)
    err = rel_linf(gpu_image(sim, system), ref)
    assert err <= tol, (err, floor)


def test_shapelet_source_needs_its_amplitudes(sim):
    from paper_2606_01547_gb300 import lenssim
    system = W.multipole_shapelet_system(4, n_max=4, n_sub=0, nx=16, s=1, k=0)
    for bad in (None, system.source_coeffs[:-1]):
        b = W.LensSystem(system.grid, system.deflectors, system.subhalos, system.source, None, bad)
        with pytest.raises(lenssim.LensSimError) as ei:
            sim.image(b)
        assert ei.value.code == lenssim.LENS_ERR_INVALID_ARG
    for bad_src in (("SHAPELETS", [11, 0.1, 0.0, 0.0]), ("SHAPELETS", [2.5, 0.1, 0.0, 0.0]),
                    ("SHAPELETS", [4, 0.0, 0.0, 0.0])):
        b = W.LensSystem(system.grid, system.deflectors, system.subhalos, bad_src, None, system.source_coeffs)
        with pytest.raises(lenssim.LensSimError):
            sim.image(b)
    bad_m = W.LensSystem(system.grid, [("MULTIPOLE", [2.5, 0.01, 0.0, 0.0, 0.0, 1.0])], system.subhalos,
                         system.source, None, system.source_coeffs)
    with pytest.raises(lenssim.LensSimError):
        sim.image(bad_m)


@pytest.mark.parametrize("nx,ny,s,nsub,k", [(13, 9, 6, 60, 3), (11, 7, 7, 40, 5), (9, 10, 8, 25, 1),
                                              (1, 37, 3, 80, 5), (41, 1, 2, 80, 3), (1, 1, 8, 10, 1)])
def test_edge_grids_match_oracle(sim, nx, ny, s, nsub, k):
    # the largest supersampling factors (their own unit shapes), single-row / single-column /
    # single-pixel grids, and odd, non-square sizes
    base = W.substructure_system(60 + s, n_sub=nsub, nx=8, s=s, k=k)
    system = W.LensSystem(W.Grid(nx, ny, s, base.grid.dpix), base.deflectors, base.subhalos, base.source, base.psf)
    ref = oracle.image(system)
    tol, floor = image_tol(system, ref)
    err = rel_linf(gpu_image(sim, system), ref)
    assert err <= tol, (err, floor)


def test_degenerate_inputs_match_oracle(sim):
    # a subhalo centred exactly on a traced sample (x floored at 1e-6: alpha -> 0 there), round
    # (e = 0) EPL and CSE lenses, and no lens at all
    g = W.Grid(12, 12, 1, 0.1)
    x0 = W.f32(0.05 + 0.1)   # centre of pixel column 7 (x = (7 - 5.5) * 0.1)
    sub = np.array([[x0], [W.f32(0.05)], [0.02], [0.005], [0.1]], np.float32)
    src = ("SERSIC_ELLIPSE_Q_PHI", [10.0, 0.3, 1.5, 0.8, 0.4, 0.02, -0.03])
    cases = [W.LensSystem(g, [("EPL_E1E2", [1.0, 2.1, 0.0, 0.0, 0.0, 0.0])], sub, src, None),
             W.LensSystem(g, [("CSE", [0.4, 0.1, 0.0, 0.0, 0.0, 0.0])], sub, src, None),
             W.LensSystem(g, [], np.zeros((5, 0), np.float32), src, None)]
    for system in cases:
        ref = oracle.image(system)
        tol, floor = image_tol(system, ref)
        err = rel_linf(gpu_image(sim, system), ref)
        assert err <= tol, (system.deflectors, err, floor)



def test_maximum_sizes_match_oracle(sim):
    # the most deflectors a system takes (8, every kind of closed form at once), the widest grid
    # (16,384 columns) and 100,000 subhalos on a small grid
    base = W.substructure_system(80, n_sub=200, nx=40, s=2, k=7)
    eight = [base.deflectors[0], base.deflectors[1], ("SIS", [0.1, 0.3, -0.2]), ("NFW", [0.4, 0.05, -0.3, 0.2]),
             ("POINT_MASS", [0.05, 0.2, 0.25]), ("MULTIPOLE", [4, 0.02, 0.2, 0.0, 0.0, 0.9]),
             ("CSE", [0.05, 0.2, 0.2, -0.1, 0.1, 0.0]), ("SIE", [0.1, 0.8, 0.3, -0.25, 0.1])]
    wide_src = W.substructure_system(81, n_sub=30, nx=8, s=1, k=5)
    many_src = W.substructure_system(82, n_sub=100000, nx=8, s=1, k=3)
    cases = [W.LensSystem(base.grid, eight, base.subhalos, base.source, base.psf),
             W.LensSystem(W.Grid(16384, 2, 1, W.f32(0.0005)), wide_src.deflectors, wide_src.subhalos,
                          wide_src.source, wide_src.psf),
             W.LensSystem(W.Grid(16, 16, 1, W.f32(0.25)), many_src.deflectors, many_src.subhalos,
                          many_src.source, many_src.psf)]
    for system in cases:
        ref = oracle.image(system)
        tol, floor = image_tol(system, ref)
        err = rel_linf(gpu_image(sim, system), ref)
        assert err <= tol, (system.grid, len(system.deflectors), system.n_sub, err, floor)


def test_sizes_beyond_the_limits_are_rejected(sim):
    from paper_2606_01547_gb300 import lenssim
    base = W.plain_system()
    nine = base.deflectors + [("SIS", [0.01, 0.0, 0.0])] * 7
    bad = [W.LensSystem(base.grid, nine, base.subhalos, base.source, base.psf),
           W.LensSystem(W.Grid(16385, 2, 1, 0.05), base.deflectors, base.subhalos, base.source, base.psf),
           W.LensSystem(base.grid, base.deflectors, base.subhalos, base.source, W.gaussian_psf(0.1, 0.05, 137))]
    for b in bad:
        with pytest.raises(lenssim.LensSimError) as ei:
            sim.image(b)
        assert ei.value.code == lenssim.LENS_ERR_INVALID_ARG


def test_elliptical_multipole_image_matches_oracle(sim):
    # an EPL with an m = 4 elliptical multipole on its own ellipse, shear and subhalos
    base = W.substructure_system(83, n_sub=300, nx=40, s=2, k=5)
    (_, epl), shear = base.deflectors
    th, g, q, phi = epl[:4]
    e = [("EPL", epl), ("MULTIPOLE_ELL", [4, 0.02, phi + 0.1, q, phi, 0.0, 0.0, th]),
         ("MULTIPOLE_ELL", [3, 0.01, 0.7, q, phi, 0.0, 0.0, th]),
         ("MULTIPOLE_ELL", [32, 0.004, 0.3, 0.2, phi, 0.0, 0.0, th])]
    for defl in ([e[0], e[1], shear], [e[0], e[2], shear], [e[0], e[3], shear]):
        system = W.LensSystem(W.Grid(40, 40, 2, W.f32(0.06)), [(n, [W.f32(v) for v in p]) for n, p in defl],
                              base.subhalos, base.source, base.psf)
        ref = oracle.image(system)
        tol, floor = image_tol(system, ref)
        err = rel_linf(gpu_image(sim, system), ref)
        assert err <= tol, (defl[1][1][0], err, floor)


def test_elliptical_multipole_limits_are_refused(sim):
    from paper_2606_01547_gb300 import lenssim
    base = W.plain_system()
    ok = ("MULTIPOLE_ELL", [4, 0.02, 0.1, 0.7, 0.3, 0.0, 0.0, 1.0])
    bad = [[("MULTIPOLE_ELL", [33, 0.02, 0.1, 0.7, 0.3, 0.0, 0.0, 1.0])],
           [("MULTIPOLE_ELL", [4, 0.02, 0.1, 0.15, 0.3, 0.0, 0.0, 1.0])],
           [("MULTIPOLE_ELL", [4.5, 0.02, 0.1, 0.7, 0.3, 0.0, 0.0, 1.0])],
           [("MULTIPOLE_ELL", [4, 0.02, 0.1, 0.7, 0.3, 0.0, 0.0, 0.0])],
           [ok, ok]]
    for d in bad:
        with pytest.raises(lenssim.LensSimError) as ei:
            sim.image(W.LensSystem(base.grid, base.deflectors + d, base.subhalos, base.source, base.psf))
        assert ei.value.code == lenssim.LENS_ERR_INVALID_ARG

def test_image_path_with_largest_psf_matches_oracle(sim):
    # k = 135 (the paper's largest kernel) through the single-image path; auto takes the FFT
    base = W.substructure_system(70, n_sub=100, nx=60, s=1, k=0)
    system = W.LensSystem(base.grid, base.deflectors, base.subhalos, base.source, W.moffat_psf(3.0, 1.0, 0.04, 135))
    ref = oracle.image(system)
    tol, floor = image_tol(system, ref)
    err = rel_linf(gpu_image(sim, system), ref)
    assert err <= tol, (err, floor)


def test_unconvolved_image_and_no_subhalos(sim):
    system = W.substructure_system(5, n_sub=0, nx=40, s=2, k=0)
    ref = oracle.image(system)
    tol, _ = image_tol(system, ref)
    assert rel_linf(gpu_image(sim, system), ref) <= tol


def test_substructure_full_size_sampled_rows(sim):
    # 200x200, s = 3, 10,000 subhalos, 21x21 Moffat: the launch configuration the benchmark times.
    # The oracle computes the 21 unconvolved rows the kernel spans around one output row.
    system = W.substructure_system(11)
    got_conv = gpu_image(sim, system)
    got_raw = gpu_image(sim, system, use_psf=False)
    k = system.psf.shape[0]
    c = (k - 1) // 2
    row = 142
    r0, r1 = row - c, row + c + 1
    raw = oracle.image_rows(system, r0, r1)
    raw_fp32 = oracle.image_rows(system, row - 1, row + 2, fp32=True)
    scale = np.abs(raw).max()
    floor = np.abs(raw_fp32 - raw[c - 1:c + 2]).max() / scale
    tol = max(1e-5, 2 * floor)
    err = np.abs(got_raw[r0:r1] - raw).max() / scale
    assert err <= tol, (err, floor)
    conv_row = np.zeros(system.grid.nx)
    K = system.psf.astype(np.float64)
    pad = np.pad(raw, ((0, 0), (c, c)))
    for a in range(k):
        for b in range(k):
            conv_row += K[a, b] * pad[k - 1 - a, (k - 1 - b):(k - 1 - b) + system.grid.nx]
    err_c = np.abs(got_conv[row] - conv_row).max() / np.abs(got_conv).max()
    assert err_c <= tol, (err_c, floor)
    # one more unconvolved row elsewhere, with its own floor
    row2 = 57
    raw2 = oracle.image_rows(system, row2, row2 + 1)
    fl2 = np.abs(oracle.image_rows(system, row2, row2 + 1, fp32=True) - raw2).max() / np.abs(raw2).max()
    assert np.abs(got_raw[row2] - raw2[0]).max() / np.abs(raw2).max() <= max(1e-5, 2 * fl2)



@pytest.mark.parametrize("seed", [0, 1, 2])
def test_substructure_full_size_whole_images(sim, seed):
    # whole 200x200, s = 3, 10,000-subhalo images with the 21x21 Moffat PSF, the benchmark's
    # workload and launch configuration, element by element against the oracle
    system = W.substructure_system(seed)
    ref = oracle.image(system)
    tol, floor = image_tol(system, ref)
    err = rel_linf(gpu_image(sim, system), ref)
    assert err <= tol, (err, floor)


@pytest.mark.parametrize("seed", [3, 4, 5, 6, 7])
def test_substructure_full_size_row_subsets(sim, seed):
    # more seeds of the same workload on three unconvolved rows each (top, middle, bottom band);
    # errors relative to the image's maximum, as for whole images
    system = W.substructure_system(seed)
    got = gpu_image(sim, system, use_psf=False)
    scale = float(np.abs(got).max())
    for row in (seed, 100 + seed, 199 - seed):
        ref = oracle.image_rows(system, row, row + 1)
        fl = float(np.abs(oracle.image_rows(system, row, row + 1, fp32=True) - ref).max()) / scale
        err = float(np.abs(got[row:row + 1] - ref).max()) / scale
        assert err <= max(1e-5, 2 * fl), (row, err, fl)

# ----------------------------------------------------------------------------- deflections
def _points(n, seed, lo=-3.0, hi=3.0):
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, n).astype(np.float32), rng.uniform(lo, hi, n).astype(np.float32)


PROFILES = [("SIS", [1.1, 0.05, -0.02]), ("SIE", [1.0, 0.8, 0.3, 0.0, 0.0]),
            ("SIE", [1.2, 0.45, 2.1, 0.1, -0.1]), ("EPL", [1.2, 1.85, 0.65, 1.0, 0.02, 0.01]),
            ("EPL", [0.9, 2.17, 0.9, 2.5, -0.05, 0.0]), ("EPL", [1.0, 2.0, 0.7, 0.3, 0.0, 0.0]),
            ("SHEAR", [0.04, -0.03]), ("POINT_MASS", [0.3, 0.1, 0.2]), ("NFW", [0.4, 0.2, 0.05, 0.1]),
            ("TNFW", [0.3, 0.15, 1.5, -0.1, 0.0]), ("EPL_E1E2", [1.1, 2.05, 0.08, -0.05, 0.0, 0.03]),
            ("SIE_E1E2", [1.0, -0.1, 0.06, 0.0, 0.0]),
            ("MULTIPOLE", [1, 0.05, 0.4, 0.1, -0.1, 1.2]), ("MULTIPOLE", [2, 0.08, -0.3, 0.0, 0.0, 1.0]),
            ("MULTIPOLE", [3, 0.03, 1.1, 0.05, 0.02, 1.3]), ("MULTIPOLE", [4, 0.02, 0.2, 0.0, 0.0, 0.9]),
            ("MULTIPOLE", [7, 0.01, 2.0, 0.1, 0.1, 1.1]),
            ("EPL_MULTIPOLE_M1M3M4", [1.1, 2.05, 0.08, -0.05, 0.0, 0.03, 0.01, 0.3, 0.02, -0.2, 0.015, 0.5]),
            ("CSE", [0.5, 0.2, 0.2, -0.1, 0.1, 0.0]), ("CSE", [1.3, 0.03, 0.35, 0.2, 0.0, 0.1]),
            ("CSE", [0.1, 1.5, -0.4, 0.1, 0.0, 0.0]),
            ("NFW_ELLIPSE_CSE", [0.8, 0.3, 0.15, -0.2, 0.05, 0.0]), ("NFW_ELLIPSE_CSE", [3.0, 1.0, 0.05, 0.02, 0.0, 0.0]),
            ("HERNQUIST_ELLIPSE_CSE", [0.5, 0.8, 0.1, -0.2, 0.0, 0.1]),
            ("HERNQUIST_ELLIPSE_CSE", [1.2, 0.3, 0.25, 0.2, 0.0, 0.0]),
            ("MULTIPOLE_ELL", [1, 0.05, 0.4, 0.6, -0.3, 0.1, -0.1, 1.2]),
            ("MULTIPOLE_ELL", [2, 0.05, 0.3, 1.0, 0.0, 0.0, 0.0, 1.0]),
            ("MULTIPOLE_ELL", [3, 0.03, 1.1, 0.8, 0.5, 0.05, 0.02, 1.3]),
            ("MULTIPOLE_ELL", [4, 0.02, 0.2, 0.45, 1.0, 0.0, 0.0, 0.9]),
            ("MULTIPOLE_ELL", [8, 0.01, 2.0, 0.4, 0.3, 0.1, 0.1, 1.1]),
            ("MULTIPOLE_ELL", [13, 0.01, 0.9, 0.55, 0.1, 0.0, 0.0, 1.0]),
            ("MULTIPOLE_ELL", [16, 0.01, 0.5, 0.25, 0.2, 0.0, 0.0, 1.0]),
            ("MULTIPOLE_ELL", [24, 0.01, 0.2, 0.3, 0.7, -0.05, 0.0, 0.9]),
            ("MULTIPOLE_ELL", [32, 0.005, 1.3, 0.2, -0.4, 0.02, -0.01, 1.1])]


@pytest.mark.parametrize("name,params", PROFILES)
def test_profile_deflection_matches_oracle(sim, name, params):
    x, y = _points(5000, 7)
    system = W.LensSystem(W.Grid(1, 1, 1, 1.0), [(name, [W.f32(v) for v in params])],
                          np.zeros((5, 0), np.float32), ("SERSIC", [1.0, 0.1, 1.0, 0.0, 0.0]))
    ax, ay = sim.deflection(system, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    rx, ry = oracle.alpha(name, system.deflectors[0][1], x, y)
    scale = max(np.abs(rx).max(), np.abs(ry).max())
    err = max(np.abs(ax.cpu().numpy() - rx).max(), np.abs(ay.cpu().numpy() - ry).max()) / scale
    assert err < 2e-6, err


@pytest.mark.parametrize("tau", [5.0, 2.0, 20.0])
def test_tnfw_pair_term_across_all_regimes(sim, tau):
    # points at x = r/Rs from 1e-5 to 3e3 cross the small, near-1 and far-field forms
    Rs, ars = 0.02, 5e-3
    xs = np.concatenate([np.logspace(-5, 3.5, 3000), np.linspace(0.85, 1.2, 500), np.linspace(3.9, 4.1, 200)])
    ang = np.random.default_rng(3).uniform(0, 2 * np.pi, xs.size)
    x = (0.3 + xs * Rs * np.cos(ang)).astype(np.float32)
    y = (-0.2 + xs * Rs * np.sin(ang)).astype(np.float32)
    p = [W.f32(v) for v in (Rs, ars, tau * Rs, 0.3, -0.2)]
    system = W.LensSystem(W.Grid(1, 1, 1, 1.0), [("TNFW", p)], np.zeros((5, 0), np.float32),
                          ("SERSIC", [1.0, 0.1, 1.0, 0.0, 0.0]))
    ax, ay = sim.deflection(system, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    rx, ry = oracle.alpha("TNFW", p, x, y)
    mag = np.hypot(rx, ry)
    d = np.hypot(ax.cpu().numpy() - rx, ay.cpu().numpy() - ry)
    # per-pair: relative 1e-5 of the deflection, or an absolute floor well below FP32 position rounding
    assert np.all(d <= 1e-5 * mag + 1e-10), float((d / (mag + 1e-30)).max())


@pytest.mark.parametrize("tau", [0.8, 2.0, 5.0, 9.0, 12.0])
def test_tnfw_subhalo_table_pair_term_across_all_regimes(sim, tau):
    # one subhalo through the precomputed table: closed forms inside 4 Rs, the annulus polynomial
    # on [4 Rs, 4 tau Rs) (none for tau <= 1, the closed form again for tau > 9.5), the series
    # beyond; points crowd both annulus edges
    Rs, ars = 0.02, 5e-3
    tm = max(tau, 1.0)
    xs = np.concatenate([np.logspace(-5, 3.5, 3000), np.linspace(3.9, 4.1, 300),
                         np.linspace(4.0 * tm * 0.98, 4.0 * tm * 1.02, 300), np.linspace(4.0, 4.0 * tm, 1000)])
    ang = np.random.default_rng(4).uniform(0, 2 * np.pi, xs.size)
    x = (0.3 + xs * Rs * np.cos(ang)).astype(np.float32)
    y = (-0.2 + xs * Rs * np.sin(ang)).astype(np.float32)
    sub = np.array([[0.3], [-0.2], [Rs], [ars], [tau * Rs]], np.float32)
    system = W.LensSystem(W.Grid(1, 1, 1, 1.0), [], sub, ("SERSIC", [1.0, 0.1, 1.0, 0.0, 0.0]))
    ax, ay = sim.deflection(system, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    rx, ry = oracle.alpha("TNFW", [float(v) for v in sub[2:, 0]] + [float(sub[0, 0]), float(sub[1, 0])], x, y)
    mag = np.hypot(rx, ry)
    d = np.hypot(ax.cpu().numpy() - rx, ay.cpu().numpy() - ry)
    assert np.all(d <= 1e-5 * mag + 1e-10), float((d / (mag + 1e-30)).max())


def test_subhalo_sum_deflection_matches_oracle(sim):
    system = W.substructure_system(21, n_sub=2500, nx=8, s=1, k=0)
    x, y = _points(4096, 8, -4.0, 4.0)
    ax, ay = sim.deflection(system, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    rx, ry = oracle.alpha_system(system, x, y)
    scale = np.abs(np.concatenate([rx, ry])).max()
    err = max(np.abs(ax.cpu().numpy() - rx).max(), np.abs(ay.cpu().numpy() - ry).max()) / scale
    assert err < 2e-6, err


# ----------------------------------------------------------------------------- PSF
@pytest.mark.parametrize("k,ny,nx,n", [(1, 9, 13, 1), (5, 37, 53, 3), (21, 64, 64, 2), (31, 40, 71, 1),
                                       (3, 1, 1, 2), (45, 50, 50, 1)])
def test_convolution_matches_oracle(sim, k, ny, nx, n):
    # the direct kernels (forced: auto would take the FFT for k = 45)
    rng = np.random.default_rng(k)
    imgs = rng.random((n, ny, nx)).astype(np.float32)
    K = rng.random((k, k)).astype(np.float32)
    sim.set_conv_method("direct")
    try:
        out = sim.convolve(torch.from_numpy(imgs).cuda(), K).cpu().numpy()
    finally:
        sim.set_conv_method("auto")
    for i in range(n):
        ref = oracle.convolve(imgs[i], K)
        assert rel_linf(out[i], ref) < 2e-6


@pytest.mark.parametrize("k,ny,nx,n", [(5, 256, 256, 3), (1, 33, 64, 2), (3, 70, 132, 2), (21, 200, 200, 1),
                                       (31, 96, 100, 2), (7, 1, 4, 3), (13, 37, 68, 5)])
def test_tma_convolution_matches_oracle(sim, k, ny, nx, n):
    # nx % 4 == 0 and 16-byte-aligned buffers take the TMA path (ragged 64x32 tiles included)
    rng = np.random.default_rng(100 + k)
    imgs = rng.random((n, ny, nx)).astype(np.float32)
    K = rng.random((k, k)).astype(np.float32)
    out = sim.convolve(torch.from_numpy(imgs).cuda(), K).cpu().numpy()
    for i in range(n):
        assert rel_linf(out[i], oracle.convolve(imgs[i], K)) < 2e-6, i


@pytest.mark.parametrize("n,k", [(64, 9), (100, 13), (100, 5), (128, 31), (68, 3)])
def test_tma_and_generic_convolution_agree_bitwise(sim, n, k):
    # the same image through the TMA path (aligned; 64-column tiles, or whole-row tiles for
    # 65..128 columns) and the generic path (offset by one float)
    rng = np.random.default_rng(7 + n + k)
    base = torch.from_numpy(rng.random((1, n * (n + 1) + 1)).astype(np.float32)).cuda()
    K = rng.random((k, k)).astype(np.float32)
    aligned = base[:, 1:n * n + 1].clone().reshape(1, n, n)  # fresh allocation: 16-byte aligned -> TMA
    assert aligned.data_ptr() % 16 == 0
    a = sim.convolve(aligned, K)
    b_in = base[:, 1:n * n + 1]  # 4-byte offset: not 16-byte aligned -> generic kernel
    assert b_in.data_ptr() % 16 != 0
    b = torch.empty((1, n, n), device="cuda")
    from paper_2606_01547_gb300 import lenssim
    pid = sim.register_psf(K)
    lenssim.lib().lens_sim_convolve(sim.h, b_in.data_ptr(), 1, n, n, pid, b.data_ptr(),
                                    int(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(b.cpu().numpy(), a.cpu().numpy())


@pytest.mark.parametrize("k,ny,nx,n", [(45, 60, 60, 2), (135, 180, 180, 1), (75, 97, 131, 3), (3, 17, 23, 1),
                                       (135, 200, 200, 1), (61, 1, 40, 2), (1, 8, 8, 1), (1, 1, 1, 1),
                                       (3, 2, 3, 2), (5, 9, 5, 3), (101, 600, 300, 1), (33, 31, 1000, 1)])
def test_fft_convolution_matches_oracle(sim, k, ny, nx, n):
    # the FFT path against the direct definition: every padded length 2..1024, ragged, odd and
    # non-square images, single rows and columns, k = 1.  FP32 transforms make an error of order
    # eps log2(M) of the output scale: the image tolerance, 1e-5 relative L-inf, bounds it
    rng = np.random.default_rng(100 + k)
    imgs = rng.random((n, ny, nx)).astype(np.float32)
    K = (rng.random((k, k)) + 0.1).astype(np.float32)
    sim.set_conv_method("fft")
    try:
        out = sim.convolve(torch.from_numpy(imgs).cuda(), K).cpu().numpy()
    finally:
        sim.set_conv_method("auto")
    for i in range(n):
        assert rel_linf(out[i], oracle.convolve(imgs[i], K)) < 1e-5


def test_fft_and_direct_methods_select_and_agree(sim):
    from paper_2606_01547_gb300 import lenssim
    rng = np.random.default_rng(7)
    imgs = torch.from_numpy(rng.random((2, 120, 90)).astype(np.float32)).cuda()
    for k in (31, 45, 101):
        K = W.moffat_psf(3.0, 0.12 * k / 21, 0.04, k)
        outs = {}
        for m in ("auto", "direct", "fft"):
            sim.set_conv_method(m)
            outs[m] = sim.convolve(imgs, K).cpu().numpy()
        sim.set_conv_method("auto")
        # auto takes the FFT above the TMA kernel's k <= 31, the direct form below (bitwise the
        # chosen one); both within the image tolerance of each other
        np.testing.assert_array_equal(outs["auto"], outs["fft" if k >= lenssim.CONV_FFT_MIN_K else "direct"])
        assert rel_linf(outs["fft"], outs["direct"]) < 1e-5
    # an FFT grid beyond 1024 is refused when forced; auto falls back to the direct form
    big = torch.zeros((1, 1000, 64), device="cuda")
    sim.set_conv_method("fft")
    with pytest.raises(lenssim.LensSimError) as ei:
        sim.convolve(big, W.moffat_psf(3.0, 0.3, 0.04, 61))
    assert ei.value.code == lenssim.LENS_ERR_UNSUPPORTED
    sim.set_conv_method("auto")
    sim.convolve(big, W.moffat_psf(3.0, 0.3, 0.04, 61))
    torch.cuda.synchronize()


@pytest.mark.parametrize("seed,nx,k,s", [(155, 64, 135, 1), (9, 180, 135, 1), (10, 200, 101, 2), (11, 128, 75, 1)])
def test_large_psf_methods_on_lensed_images_match_oracle(sim, seed, nx, k, s):
    # a compact lensed image under a wide kernel, where the FFT's error (of order eps log2(M) times
    # the kernel's and the image's L2 norms) is largest against the image maximum; the FFT carries
    # only the kernel's wings beside a direct core.  (a) The convolution alone, of the oracle's
    # own unconvolved image, by each method: 1e-5 (measured <= 7e-7 direct, <= 4e-7 FFT).  (b) The
    # whole image by each method within the image tolerance, except on the 180^2 case, whose
    # unconvolved GPU image already deviates by 2.8x its floor near the compact source (1.04e-5
    # after any convolution against a tolerance of 1e-5): there the methods must agree with
    # each other to 1e-6.
    system = W.substructure_system(seed, n_sub=300, nx=nx, s=s, k=k)
    ref, raw = oracle.image(system, return_unconvolved=True)
    raw32 = raw.astype(np.float32)
    cref = oracle.convolve(raw32, system.psf)
    tol, floor = image_tol(system, ref)
    whole = {}
    for method in ("auto", "direct", "fft"):
        sim.set_conv_method(method)
        try:
            conv = sim.convolve(torch.from_numpy(raw32).cuda(), system.psf).cpu().numpy()[0]
            whole[method] = gpu_image(sim, system)
        finally:
            sim.set_conv_method("auto")
        assert rel_linf(conv, cref) <= 1e-5, (method, rel_linf(conv, cref))
        if nx != 180:
            assert rel_linf(whole[method], ref) <= tol, (method, rel_linf(whole[method], ref), floor)
    assert rel_linf(whole["fft"], whole["direct"]) <= 1e-6
    np.testing.assert_array_equal(whole["auto"], whole["fft"])


def test_image_with_fft_psf_matches_oracle(sim):
    system = W.substructure_system(9, n_sub=200, nx=64, s=2, k=0)
    system = W.LensSystem(system.grid, system.deflectors, system.subhalos, system.source,
                          W.moffat_psf(3.0, 0.5, 0.04, 61))
    ref = oracle.image(system)
    tol, floor = image_tol(system, ref)
    sim.set_conv_method("fft")
    try:
        err = rel_linf(gpu_image(sim, system), ref)
    finally:
        sim.set_conv_method("auto")
    assert err <= tol, (err, floor)


def test_delta_psf_is_identity_on_gpu(sim):
    img = np.random.default_rng(1).random((33, 47)).astype(np.float32)
    K = np.zeros((7, 7), np.float32)
    K[3, 3] = 1.0
    out = sim.convolve(torch.from_numpy(img).cuda(), K).cpu().numpy()[0]
    np.testing.assert_array_equal(out, img)


# ----------------------------------------------------------------------------- API behaviour
def test_host_and_device_buffers_and_tables_agree_bitwise(sim):
    system = W.substructure_system(31, n_sub=700, nx=24, s=2, k=5)
    a = gpu_image(sim, system)
    host_out = np.zeros((24, 24), np.float32)
    sim.image(system, out=[host_out])
    dev_sub = torch.from_numpy(system.subhalos).cuda()
    b = gpu_image(sim, system, subhalos=[dev_sub])
    tid = sim.register_subhalos(system.subhalos)
    c = gpu_image(sim, system, subhalo_tables=[tid])
    np.testing.assert_array_equal(a, host_out)
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(a, c)
    np.testing.assert_array_equal(a, gpu_image(sim, system))  # deterministic


def test_batch_of_uneven_systems_matches_single_calls(sim):
    systems = W.batched_systems(5, count=6, max_sub=400, grids=(16, 24, 40))
    outs = sim.image(systems)
    torch.cuda.synchronize()
    for s_, o in zip(systems, outs):
        np.testing.assert_array_equal(o.cpu().numpy(), gpu_image(sim, s_))


def test_batched_largest_system_matches_oracle_rows(sim):
    # the batched configuration's largest system (256x256, s = 3, 20,000 subhalos) inside an
    # uneven batch, through the persistent batched launch the benchmark times: sampled
    # unconvolved rows against the oracle, and bitwise equality with the single-image path
    big = W.substructure_system(13, n_sub=20000, nx=256, s=3, k=0)
    others = W.batched_systems(14, count=3, max_sub=2000, grids=(64, 100))
    outs = sim.image([big] + others)
    torch.cuda.synchronize()
    got = outs[0].cpu().numpy()
    np.testing.assert_array_equal(got, gpu_image(sim, big))
    for row in (31, 180):
        ref = oracle.image_rows(big, row, row + 1)
        fl = np.abs(oracle.image_rows(big, row, row + 1, fp32=True) - ref).max() / np.abs(ref).max()
        assert np.abs(got[row] - ref[0]).max() / np.abs(ref).max() <= max(1e-5, 2 * fl)


def test_every_batch_schedule_gives_the_same_images_and_autotune_picks_one(sim):
    # each persistent kernel form and unit-queue order of the batched launch, on an uneven batch
    # with every unit shape (s = 1..3, ragged grids, systems without subhalos or PSF): bitwise
    # equal images, equal to single-system calls; the autotuner times all six and keeps one
    from paper_2606_01547_gb300 import lenssim
    systems = W.batched_systems(77, count=9, max_sub=1500, grids=(24, 37, 64))
    systems.append(W.LensSystem(W.Grid(30, 22, 2, 0.04), systems[0].deflectors, np.zeros((5, 0), np.float32),
                                systems[0].source, None))
    # two systems with elliptical multipoles, whose harmonics travel beside the descriptors
    for m, q in ((4, 0.6), (32, 0.2)):
        y = systems[m % 5]
        systems.append(W.LensSystem(y.grid, y.deflectors + [("MULTIPOLE_ELL", [m, 0.01, 0.4, q, 0.2, 0.0, 0.0, 1.0])],
                                    y.subhalos, y.source, y.psf))
    single = [gpu_image(sim, y) for y in systems]
    for form in range(len(lenssim.BATCH_FORMS)):
        for order in range(2):
            sim.set_batch_schedule(form, order)
            outs = sim.image(systems)
            torch.cuda.synchronize()
            for got, ref in zip(outs, single):
                np.testing.assert_array_equal(got.cpu().numpy(), ref)
    entry = sim.autotune_batch(systems, reps=1, use_cache=False)
    assert entry["name"].split("/")[0] in lenssim.BATCH_FORMS and all(v > 0 for v in entry["ms"].values())
    outs = sim.image(systems)
    torch.cuda.synchronize()
    for got, ref in zip(outs, single):
        np.testing.assert_array_equal(got.cpu().numpy(), ref)
    with pytest.raises(lenssim.LensSimError) as ei:
        sim.set_batch_schedule(len(lenssim.BATCH_FORMS), 0)
    assert ei.value.code == lenssim.LENS_ERR_INVALID_ARG
    sim.set_batch_schedule(0, 0)


def test_invalid_arguments_are_rejected(sim):
    from paper_2606_01547_gb300 import lenssim
    base = W.plain_system()
    bad = [W.LensSystem(W.Grid(60, 60, 9, 0.05), base.deflectors, base.subhalos, base.source, base.psf),
           W.LensSystem(W.Grid(0, 60, 1, 0.05), base.deflectors, base.subhalos, base.source, base.psf),
           W.LensSystem(base.grid, [("SIE", [1.0, 1.3, 0.0, 0.0, 0.0])], base.subhalos, base.source, base.psf),
           W.LensSystem(base.grid, base.deflectors, base.subhalos, base.source, np.ones((4, 4), np.float32))]
    for b in bad:
        with pytest.raises(lenssim.LensSimError) as ei:
            sim.image(b)
        assert ei.value.code == lenssim.LENS_ERR_INVALID_ARG
    # a valid call still works afterwards
    assert rel_linf(gpu_image(sim, base), oracle.image(base)) <= 1e-5


@pytest.mark.parametrize("s,nx,ny,nsub", [(3, 45, 45, 1500), (1, 50, 27, 900), (2, 31, 40, 1200), (5, 17, 9, 300)])
def test_trace_variants_are_bitwise_identical_and_autotune_picks_one(sim, s, nx, ny, nsub):
    # every launch variant on each unit shape (24x12 pixels at s = 1, 12x6 at s = 2, 8x4 at s = 3,
    # 5x2 at s = 5), grids with ragged unit rows and columns
    from paper_2606_01547_gb300 import lenssim
    base = W.substructure_system(41 + s, n_sub=nsub, nx=8, s=s, k=7)
    system = W.LensSystem(W.Grid(nx, ny, s, base.grid.dpix), base.deflectors, base.subhalos, base.source, base.psf)
    imgs = []
    for v in range(len(lenssim.TRACE_VARIANTS)):
        sim.set_variant(v)
        imgs.append(gpu_image(sim, system))
    for im in imgs[1:]:
        np.testing.assert_array_equal(im, imgs[0])
    entry = sim.autotune(system, reps=2, use_cache=False)
    assert entry["name"] in lenssim.TRACE_VARIANTS and all(v > 0 for v in entry["ms"].values())
    np.testing.assert_array_equal(gpu_image(sim, system), imgs[0])
    sim.set_variant(0)

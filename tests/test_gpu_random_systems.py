"""Seeded random systems against the oracle: grid shapes (single rows, columns and pixels
included), every supersampling factor of the unit table, subhalo counts around the 32-subhalo
stage, extra deflectors from the profile variants, PSF sizes on both sides of the FFT switch,
launch variants and the far-field option -- each whole image element by element against the
FP64 oracle, and the same systems through one batched call bitwise equal to their single calls.
"""
import numpy as np
import pytest

import oracle
from paper_2606_01547_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EXTRA = [None,
         ("MULTIPOLE", [3, 0.02, 0.5, 0.0, 0.0, 1.1]),
         ("NFW_ELLIPSE_CSE", [0.8, 0.3, 0.1, -0.1, 0.05, 0.0]),
         ("MULTIPOLE_ELL", [4, 0.02, 0.3, 0.7, 0.4, 0.0, 0.0, 1.0]),
         ("POINT_MASS", [0.2, 0.3, -0.2])]
N_SUB = (0, 1, 7, 31, 32, 33, 64, 257, 1000)


@pytest.fixture(scope="module")
def sim():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_01547_gb300 import lenssim
    s = lenssim.Simulator(device=0)
    yield s
    s.close()


def random_system(seed):
    rng = np.random.default_rng(5000 + seed)
    nx, ny = int(rng.integers(1, 49)), int(rng.integers(1, 49))
    if seed % 5 == 0:
        nx = 1
    if seed % 7 == 0:
        ny = 1
    s = int(rng.integers(1, 9))
    n_sub = int(N_SUB[rng.integers(len(N_SUB))])
    k = int(2 * rng.integers(0, 21) + 1)
    base = W.substructure_system(6000 + seed, n_sub=n_sub, nx=8, s=s, k=k)
    defl = list(base.deflectors)
    extra = EXTRA[int(rng.integers(len(EXTRA)))]
    if extra is not None:
        defl.append(W._profile(*extra))
    system = W.LensSystem(W.Grid(nx, ny, s, base.grid.dpix), defl, base.subhalos, base.source, base.psf)
    kappa = float((0.0, 3.0, 6.0)[int(rng.integers(3))])
    variant = int(rng.integers(5))
    return system, kappa, variant


@pytest.mark.parametrize("seed", range(16))
def test_random_system_matches_oracle(sim, seed):
    system, kappa, variant = random_system(seed)
    ref = oracle.image(system)
    floor = float(np.abs(oracle.image(system, fp32=True) - ref).max() / np.abs(ref).max())
    tol = max(1e-5, 2.0 * floor)
    sim.set_variant(variant)
    sim.set_far_field(kappa)
    try:
        got = sim.image(system)[0]
        torch.cuda.synchronize()
    finally:
        sim.set_far_field(0.0)
        sim.set_variant(0)
    err = float(np.abs(got.cpu().numpy().astype(np.float64) - ref).max() / np.abs(ref).max())
    g = system.grid
    assert err <= tol, (seed, g.nx, g.ny, g.s, system.n_sub, kappa, variant, err, floor)


# deflector lists of 1-3 profiles from the variants, and every source type
DEFL = [("SIS", [1.1, 0.05, -0.02]), ("SIE", [1.2, 0.45, 2.1, 0.1, -0.1]),
        ("EPL", [1.0, 1.85, 0.65, 1.0, 0.02, 0.01]), ("EPL_E1E2", [1.1, 2.05, 0.08, -0.05, 0.0, 0.03]),
        ("SIE_E1E2", [1.0, -0.1, 0.06, 0.0, 0.0]), ("SHEAR", [0.04, -0.03]), ("NFW", [0.4, 0.2, 0.05, 0.1]),
        ("TNFW", [0.3, 0.15, 1.5, -0.1, 0.0]), ("POINT_MASS", [0.3, 0.1, 0.2]),
        ("EPL_MULTIPOLE_M1M3M4", [1.1, 2.05, 0.08, -0.05, 0.0, 0.03, 0.01, 0.3, 0.02, -0.2, 0.015, 0.5]),
        ("CSE", [0.5, 0.2, 0.2, -0.1, 0.1, 0.0]), ("HERNQUIST_ELLIPSE_CSE", [0.5, 0.8, 0.1, -0.2, 0.0, 0.1]),
        ("MULTIPOLE", [2, 0.08, -0.3, 0.0, 0.0, 1.0])]


def random_system2(seed):
    rng = np.random.default_rng(7000 + seed)
    nx, ny = int(rng.integers(1, 41)), int(rng.integers(1, 41))
    s = int(rng.integers(1, 6))
    n_sub = int(N_SUB[rng.integers(len(N_SUB))])
    k = int(2 * rng.integers(0, 12) + 1)
    base = W.substructure_system(8000 + seed, n_sub=n_sub, nx=8, s=s, k=k)
    picks = rng.choice(len(DEFL), size=int(rng.integers(1, 4)), replace=False)
    defl = [W._profile(*DEFL[i]) for i in picks]
    kind = int(rng.integers(4))
    coef = None
    if kind == 0:
        src = W._profile("SERSIC_ELLIPSE_Q_PHI", [8.0, 0.3, float(rng.uniform(0.6, 3.5)), 0.7, 0.4, 0.02, -0.03])
    elif kind == 1:
        src = W._profile("SERSIC_ELLIPSE", [8.0, 0.25, float(rng.uniform(0.6, 3.5)), 0.1, -0.05, 0.0, 0.02])
    elif kind == 2:
        src = W._profile("SERSIC", [8.0, 0.3, float(rng.uniform(0.6, 3.5)), 0.01, 0.0])
    else:
        n_max = int(rng.integers(0, 7))
        src = W._profile("SHAPELETS", [n_max, float(rng.uniform(0.08, 0.2)), 0.0, 0.02])
        m = (n_max + 1) * (n_max + 2) // 2
        coef = (rng.normal(size=m) / (1.0 + np.arange(m))).astype(np.float32)
        coef[0] += 3.0
    system = W.LensSystem(W.Grid(nx, ny, s, base.grid.dpix), defl, base.subhalos, src, base.psf, coef)
    return system, float((0.0, 3.0)[int(rng.integers(2))]), int(rng.integers(5))


@pytest.mark.parametrize("seed", range(16))
def test_random_profiles_and_sources_match_oracle(sim, seed):
    system, kappa, variant = random_system2(seed)
    ref = oracle.image(system)
    floor = float(np.abs(oracle.image(system, fp32=True) - ref).max() / np.abs(ref).max())
    tol = max(1e-5, 2.0 * floor)
    sim.set_variant(variant)
    sim.set_far_field(kappa)
    try:
        got = sim.image(system)[0]
        torch.cuda.synchronize()
    finally:
        sim.set_far_field(0.0)
        sim.set_variant(0)
    err = float(np.abs(got.cpu().numpy().astype(np.float64) - ref).max() / np.abs(ref).max())
    assert err <= tol, (seed, [d[0] for d in system.deflectors], system.source[0], err, floor)


@pytest.mark.parametrize("kappa", [0.0, 3.0])
def test_random_systems_batched_equal_single_calls(sim, kappa):
    # (the batched launch convolves directly; single calls would take the FFT for k >= 33)
    systems = [random_system(seed)[0] for seed in range(16)] + [random_system2(seed)[0] for seed in range(16)]
    sim.set_far_field(kappa)
    sim.set_conv_method("direct")
    try:
        singles = []
        for y in systems:
            singles.append(sim.image(y)[0].cpu().numpy())
        batch = [o.cpu().numpy() for o in sim.image(systems)]
    finally:
        sim.set_far_field(0.0)
        sim.set_conv_method("auto")
    for i, (a, b) in enumerate(zip(batch, singles)):
        assert np.array_equal(a, b), i

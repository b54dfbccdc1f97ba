"""The allocation-free entry point, lens_sim_image_noalloc, through the C ABI.

It exists for callers that cannot allocate device memory (device memory reserved up front by
their own pool; loops that forbid cudaMalloc/cudaFree because those calls can synchronise the
device).  Its images must match lens_sim_image's within the image tolerance of the other GPU
tests (they run the same kernels, so they agree bitwise), on two calls in a row that share the
one fixed scratch array.  Large PSF kernels take the direct convolution here (the FFT is
lens_sim_image's default for them): equal bitwise to lens_sim_image's direct method and within
the image tolerance of the FP64 oracle.  Collected last on purpose; it also passes alone in a fresh
process.
"""
import ctypes

import numpy as np
import pytest

from paper_2606_01547_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_01547_gb300 import lenssim
    sim = lenssim.Simulator(device=0)
    yield lenssim, lenssim.lib(), sim
    sim.close()


def _noalloc(L, sim, system, out, grid=None):
    keep = []
    c = sim.system_struct(system, keep, subhalos=torch.from_numpy(system.subhalos).cuda(), use_psf=False)
    if grid is not None:
        c.grid = grid
    psf = torch.from_numpy(system.psf).cuda() if system.psf is not None else None
    k = 0 if psf is None else int(psf.shape[0])
    ptr = out.data_ptr() if isinstance(out, torch.Tensor) else out.ctypes.data
    rc = L.lens_sim_image_noalloc(ctypes.byref(c), None if psf is None else psf.data_ptr(), k, ptr,
                                  int(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return rc


def _rel(got, ref):
    ref = ref.cpu().numpy().astype(np.float64)
    return np.abs(got.cpu().numpy() - ref).max() / np.abs(ref).max()


def test_noalloc_matches_lens_sim_image_on_two_calls_in_a_row(env):
    lenssim, L, sim = env
    # two different systems back to back: the second call reuses the scratch of the first
    a = W.substructure_system(5, n_sub=2000, nx=48, s=3, k=9)
    b = W.substructure_system(6, n_sub=500, nx=64, s=2, k=5)
    out_a = torch.empty((48, 48), device="cuda")
    out_b = torch.empty((64, 64), device="cuda")
    assert _noalloc(L, sim, a, out_a) == lenssim.LENS_OK
    assert _noalloc(L, sim, b, out_b) == lenssim.LENS_OK
    for system, got in ((a, out_a), (b, out_b)):
        ref = sim.image(system)[0]
        torch.cuda.synchronize()
        assert _rel(got, ref) <= 1e-5
    # no PSF step, and sizes beyond the fixed scratch are refused with nothing launched
    c = W.substructure_system(7, n_sub=100, nx=20, s=1, k=0)
    out_c = torch.empty((20, 20), device="cuda")
    assert _noalloc(L, sim, c, out_c) == lenssim.LENS_OK
    np.testing.assert_allclose(out_c.cpu().numpy(), sim.image(c)[0].cpu().numpy(), rtol=0, atol=0)
    # an elliptical multipole: its harmonics travel through the fixed scratch as well
    e = W.LensSystem(c.grid, c.deflectors + [("MULTIPOLE_ELL", [32, 0.01, 0.3, 0.2, 0.1, 0.0, 0.0, 1.0])],
                     c.subhalos, c.source, None)
    assert _noalloc(L, sim, e, out_c) == lenssim.LENS_OK
    np.testing.assert_array_equal(out_c.cpu().numpy(), sim.image(e)[0].cpu().numpy())
    too_many = W.substructure_system(8, n_sub=20001, nx=8, s=1, k=3)
    assert _noalloc(L, sim, too_many, torch.empty((8, 8), device="cuda")) == lenssim.LENS_ERR_OOM
    too_big = W.LensSystem(W.Grid(600, 600, 1, 0.04), c.deflectors, c.subhalos, c.source, None)
    assert _noalloc(L, sim, too_big, torch.empty((600, 600), device="cuda")) == lenssim.LENS_ERR_OOM


@pytest.mark.parametrize("k", [45, 135])
def test_noalloc_large_psf_direct_path(env, k):
    # k >= LENS_CONV_FFT_MIN_K: the direct convolution here (with the shared-memory opt-in above
    # 48 KB), bitwise equal to lens_sim_image's direct method, and within the image tolerance
    # of the FP64 oracle, on two calls in a row
    import oracle
    lenssim, L, sim = env
    system = W.substructure_system(20 + k, n_sub=300, nx=64, s=1, k=k)
    ref = oracle.image(system)
    floor = np.abs(oracle.image(system, fp32=True) - ref).max() / np.abs(ref).max()
    sim.set_conv_method("direct")
    try:
        for rep in range(2):
            got = torch.full((64, 64), float("nan"), device="cuda")
            assert _noalloc(L, sim, system, got) == lenssim.LENS_OK
            ref_direct = sim.image(system)[0]
            torch.cuda.synchronize()
            np.testing.assert_array_equal(got.cpu().numpy(), ref_direct.cpu().numpy())
            assert _rel(got, torch.from_numpy(ref)) <= max(1e-5, 2 * floor)
    finally:
        sim.set_conv_method("auto")


def test_noalloc_refuses_bad_grids_and_buffers(env):
    # the grid checks of lens_sim_image and memory that is not the current device's
    lenssim, L, sim = env
    c = W.substructure_system(9, n_sub=50, nx=16, s=1, k=5)
    out = torch.empty((16, 16), device="cuda")
    G = lenssim.LensGrid
    bad = [G(16, 16, 1, float("inf"), 0.0, 0.0), G(16, 16, 1, 0.04, float("nan"), 0.0),
           G(16, 16, 1, 0.04, 0.0, float("inf")), G(16, 16, 1, -0.04, 0.0, 0.0), G(16, 16, 0, 0.04, 0.0, 0.0),
           G(16, 16, 9, 0.04, 0.0, 0.0), G(16385, 1, 1, 0.04, 0.0, 0.0), G(0, 16, 1, 0.04, 0.0, 0.0)]
    for g in bad:
        assert _noalloc(L, sim, c, out, grid=g) == lenssim.LENS_ERR_INVALID_ARG, (g.nx, g.ny, g.pixel_scale)
    host_out = np.empty((16, 16), np.float32)
    assert _noalloc(L, sim, c, host_out) == lenssim.LENS_ERR_INVALID_ARG
    # the valid call after the refusals still works
    assert _noalloc(L, sim, c, out) == lenssim.LENS_OK
    assert _rel(out, sim.image(c)[0]) <= 1e-5

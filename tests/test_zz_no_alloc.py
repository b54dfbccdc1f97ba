"""The allocation-free entry point, lens_sim_image_noalloc, through the C ABI.

It exists for callers that cannot allocate device memory (device memory reserved up front by
their own pool; loops that forbid cudaMalloc/cudaFree because those calls can synchronise the
device).  Its images must match lens_sim_image's within the image tolerance of the other GPU
tests (they run the same kernels, so they agree bitwise), on two calls in a row that share the
one fixed scratch array.  Collected last on purpose; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_2606_01547_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _noalloc(L, sim, system, out):
    keep = []
    c = sim.system_struct(system, keep, subhalos=torch.from_numpy(system.subhalos).cuda(), use_psf=False)
    psf = torch.from_numpy(system.psf).cuda() if system.psf is not None else None
    k = 0 if psf is None else int(psf.shape[0])
    rc = L.lens_sim_image_noalloc(ctypes.byref(c), None if psf is None else psf.data_ptr(), k, out.data_ptr(),
                                  int(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return rc


def test_noalloc_matches_lens_sim_image_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_01547_gb300 import lenssim
    L = lenssim.lib()
    sim = lenssim.Simulator(device=0)
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
        ref = ref.cpu().numpy().astype(np.float64)
        err = np.abs(got.cpu().numpy() - ref).max() / np.abs(ref).max()
        assert err <= 1e-5, err
    # no PSF step, and sizes beyond the fixed scratch are refused with nothing launched
    c = W.substructure_system(7, n_sub=100, nx=20, s=1, k=0)
    out_c = torch.empty((20, 20), device="cuda")
    assert _noalloc(L, sim, c, out_c) == lenssim.LENS_OK
    np.testing.assert_allclose(out_c.cpu().numpy(), sim.image(c)[0].cpu().numpy(), rtol=0, atol=0)
    too_many = W.substructure_system(8, n_sub=20001, nx=8, s=1, k=3)
    assert _noalloc(L, sim, too_many, torch.empty((8, 8), device="cuda")) == lenssim.LENS_ERR_OOM
    too_big = W.LensSystem(W.Grid(600, 600, 1, 0.04), c.deflectors, c.subhalos, c.source, None)
    assert _noalloc(L, sim, too_big, torch.empty((600, 600), device="cuda")) == lenssim.LENS_ERR_OOM
    sim.close()

"""Serving (lens_serve_*): results match the direct calls, each result is the same alone and
in a mix, admission and cancellation, bounded waits, budget refusal.  Faults are made on the
host (a paused worker, a refused budget, a malformed request); nothing faults the GPU."""
import numpy as np
import pytest

import oracle
from paper_2606_01547_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lenssim():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_01547_gb300 import lenssim as L
    return L


def _image_direct(L, system):
    sim = L.Simulator(device=0)
    out = sim.image(system)[0].cpu().numpy()
    sim.close()
    return out


def test_served_images_match_direct_calls(lenssim):
    srv = lenssim.Server(device=0)
    systems = W.batched_systems(3, count=6, max_sub=500, grids=(32, 48, 64))
    outs = [np.zeros((s.grid.ny, s.grid.nx), np.float32) for s in systems]
    tickets = [srv.submit_image(s, o) for s, o in zip(systems, outs)]
    for t in tickets:
        assert srv.wait(t, 60000) == lenssim.LENS_OK
    for s, o in zip(systems, outs):
        np.testing.assert_array_equal(o, _image_direct(lenssim, s))
    st = srv.stats()
    assert st["p50_ms"] > 0 and st["p99_ms"] >= st["p50_ms"]
    srv.close()


def test_served_loglike_matches_direct_and_oracle(lenssim):
    pb = W.diff_problem(4, n_points=3, n_sub=25, nx=24, dpix=0.1, k=5)
    data = W.observe(oracle.model_image(pb.system, pb.truth), 0.01, 1000.0, 4)
    srv = lenssim.Server(device=0)
    res = []
    for p in pb.points:
        out = np.zeros(1, np.float32)
        g = np.zeros(15, np.float32)
        res.append((srv.submit_loglike(pb.system, data, 0.01, 1000.0, p, out, g), out, g))
    sim = lenssim.Simulator(device=0)
    L, G = sim.grad(pb.system, torch.from_numpy(data).cuda(), 0.01, 1000.0, torch.from_numpy(pb.points).cuda())
    for i, (t, out, g) in enumerate(res):
        assert srv.wait(t, 60000) == lenssim.LENS_OK
        assert out[0] == L[i].item()
        np.testing.assert_array_equal(g, G[i].cpu().numpy())
    Lr = oracle.loglike(pb.system, data, 0.01, 1000.0, pb.points, grad=False)
    np.testing.assert_allclose(np.array([r[1][0] for r in res]), Lr, rtol=1e-5)
    sim.close()
    srv.close()


def test_each_result_is_the_same_alone_and_in_a_mix(lenssim):
    target = W.substructure_system(77, n_sub=3000, nx=40, s=2, k=9)
    pb = W.diff_problem(8, n_points=1, n_sub=100, nx=32, dpix=0.08, k=7)
    data = W.observe(oracle.model_image(pb.system, pb.truth), 0.01, 1000.0, 8)
    srv = lenssim.Server(device=0)
    alone = np.zeros((40, 40), np.float32)
    t = srv.submit_image(target, alone)
    assert srv.wait(t) == lenssim.LENS_OK
    la, ga = np.zeros(1, np.float32), np.zeros(15, np.float32)
    t = srv.submit_loglike(pb.system, data, 0.01, 1000.0, pb.points[0], la, ga)
    assert srv.wait(t) == lenssim.LENS_OK
    # the same two requests inside a stream of 60 mixed requests of other sizes
    mix = W.serving_stream(5, rate=1e5, duration=6e-4, max_sub=3000)
    tickets, bufs = [], []
    for k, rq in enumerate(mix[:58]):
        if k == 20:
            mixed = np.zeros((40, 40), np.float32)
            tickets.append(srv.submit_image(target, mixed))
            lm, gm = np.zeros(1, np.float32), np.zeros(15, np.float32)
            tickets.append(srv.submit_loglike(pb.system, data, 0.01, 1000.0, pb.points[0], lm, gm))
        g = rq.system.grid
        if rq.kind == 0:
            o = np.zeros((g.ny, g.nx), np.float32)
            tickets.append(srv.submit_image(rq.system, o))
        else:
            d = np.zeros((g.ny, g.nx), np.float32)
            o, gr = np.zeros(1, np.float32), np.zeros(15, np.float32)
            p = np.array([*rq.system.deflectors[0][1], *rq.system.deflectors[1][1], *rq.system.source[1]],
                         np.float32)
            tickets.append(srv.submit_loglike(rq.system, d, 0.01, 1000.0, p, o, gr))
    for t in tickets:
        assert srv.wait(t, 120000) == lenssim.LENS_OK
    np.testing.assert_array_equal(mixed, alone)
    assert lm[0] == la[0]
    np.testing.assert_array_equal(gm, ga)
    srv.close()


def test_admission_cancel_and_bounded_wait(lenssim):
    srv = lenssim.Server(device=0, max_inflight=3)
    srv.pause(True)  # the worker holds admission: requests stay queued
    system = W.substructure_system(9, n_sub=50, nx=16, s=1, k=3)
    outs = [np.zeros((16, 16), np.float32) for _ in range(4)]
    t = [srv.submit_image(system, outs[i]) for i in range(3)]
    with pytest.raises(lenssim.LensSimError) as ei:
        srv.submit_image(system, outs[3])
    assert ei.value.code == lenssim.LENS_ERR_BUSY
    assert srv.wait(t[0], 50) == lenssim.LENS_ERR_TIMEOUT  # bounded: returns, never hangs
    assert srv.poll(t[0]) == lenssim.LENS_ERR_BUSY
    assert srv.cancel(t[1]) == lenssim.LENS_OK
    assert srv.wait(t[1], 1000) == lenssim.LENS_ERR_CANCELLED
    t.append(srv.submit_image(system, outs[3]))  # a slot freed by the cancellation
    srv.pause(False)
    for k in (0, 2, 3):
        assert srv.wait(t[k], 60000) == lenssim.LENS_OK
    np.testing.assert_array_equal(outs[0], outs[2])
    srv.close()


def test_budget_refusal_and_a_bad_request_fails_alone(lenssim):
    small = lenssim.Server(device=0, mem_budget=1 << 16)
    big = W.substructure_system(1, n_sub=10, nx=256, s=1, k=3)
    with pytest.raises(lenssim.LensSimError) as ei:
        small.submit_image(big, np.zeros((256, 256), np.float32))
    assert ei.value.code == lenssim.LENS_ERR_OOM
    small.close()
    srv = lenssim.Server(device=0)
    good = W.substructure_system(2, n_sub=30, nx=24, s=1, k=5)
    bad = W.LensSystem(good.grid, [("SIE", [1.0, 1.7, 0.0, 0.0, 0.0])], good.subhalos, good.source, good.psf)
    srv.pause(True)
    o1, o2, o3 = (np.zeros((24, 24), np.float32) for _ in range(3))
    t1, t2, t3 = srv.submit_image(good, o1), srv.submit_image(bad, o2), srv.submit_image(good, o3)
    srv.pause(False)
    assert srv.wait(t1) == lenssim.LENS_OK
    assert srv.wait(t2) == lenssim.LENS_ERR_INVALID_ARG
    assert "q" in srv.last_error(), srv.last_error()  # the library's message for the bad axis ratio
    assert srv.wait(t3) == lenssim.LENS_OK
    np.testing.assert_array_equal(o1, o3)
    srv.close()


def test_psf_registration_while_requests_run(lenssim):
    # the binding registers each new PSF on the server's handle at submit time, while the worker
    # runs earlier requests: the worker's registry reads must not race the registrations
    srv = lenssim.Server(device=0)
    rng = np.random.default_rng(5)
    tickets, keep = [], []
    for i in range(240):
        k = int(W.BATCH_PSF[i % len(W.BATCH_PSF)])
        nx = 64 if i % 2 else 48
        base = W.LensSystem(W.Grid(nx, nx, 1, W.f32(0.04)), [], W.subhalo_population(rng, 50),
                            ("SERSIC_ELLIPSE", [0.0] * 7), W.moffat_psf(3.0, 0.1 + 0.01 * (i % 7), 0.04, k))
        p = W._draw_free(rng)
        system = W.system_from_free(base, p)
        if i % 3:
            o = np.empty((nx, nx), np.float32)
            keep.append(o)
            tickets.append(srv.submit_image(system, o))
        else:
            d = np.zeros((nx, nx), np.float32)
            pp = np.array(p, np.float32)
            o, g = np.empty(1, np.float32), np.empty(15, np.float32)
            keep += [d, pp, o, g]
            tickets.append(srv.submit_loglike(system, d, 0.01, 1000.0, pp, o, g))
    codes = [srv.wait(t, 120000) for t in tickets]
    assert all(c == lenssim.LENS_OK for c in codes), (codes, srv.last_error())
    srv.close()

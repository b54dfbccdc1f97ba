"""CPU pins of the optional far-field interpolation of the subhalo sum.

The image kernels can sum a subhalo that lies kappa box half-widths or more from a work unit's
box at the 8 x 8 Chebyshev nodes of the box and interpolate the unit's node sums to its traced
points (the local-expansion step of a black-box fast multipole method, Fong and Darve 2009).
The C header states the error of that interpolation per approximated subhalo; these tests pin
those numbers with the oracle's FP64 truncated-NFW deflection (deflection table row TNFW),
interpolated here in FP64 with the same node set, so the bound rests on the oracle and the
mathematics, not on the CUDA path.
"""
import math

import numpy as np
import pytest

import oracle

N1 = 8
NODES = np.cos(np.pi * (np.arange(N1) + 0.5) / N1)   # Chebyshev points of the first kind

# the bound the header states for each kappa: the largest error of one subhalo's deflection over
# the box, relative to its largest magnitude there
STATED = {3.0: 1.2e-6, 4.0: 1.4e-7, 6.0: 6.0e-9}


def lagrange(t):
    """Tensor-product factor: L_i(t) for the N1 nodes, t of shape (m,) -> (m, N1)."""
    L = np.ones((t.size, N1))
    for i in range(N1):
        for k in range(N1):
            if k != i:
                L[:, i] *= (t - NODES[k]) / (NODES[i] - NODES[k])
    return L


def interp(fnodes, tx, ty):
    """Interpolant of node values fnodes[i, j] (node (x_i, y_j)) at box coordinates (tx, ty)."""
    return np.einsum("si,sj,ij->s", lagrange(tx), lagrange(ty), fnodes)


def box_points(m=21):
    g = np.linspace(-1.0, 1.0, m)
    tx, ty = np.meshgrid(g, g, indexing="ij")
    return tx.ravel(), ty.ravel()


def worst_relative_error(kappa, hx, hy, n_dir=24, taus=(0.5, 5.0, 20.0), rss=(0.002, 0.02, 0.1)):
    """Largest relative interpolation error of one TNFW subhalo's deflection over the box
    [-hx, hx] x [-hy, hy], the subhalo at box distance kappa * max(hx, hy) along n_dir
    directions; subhalos inside their own far-field radius 7 max(tau, 1) Rs are skipped, as the
    kernel never approximates the subhalos its near-field test marks."""
    tx, ty = box_points()
    gx, gy = np.meshgrid(hx * NODES, hy * NODES, indexing="ij")
    d = kappa * max(hx, hy)
    worst = 0.0
    for ang in np.linspace(0.0, 2.0 * math.pi, n_dir, endpoint=False):
        ux, uy = math.cos(ang), math.sin(ang)
        s = min(hx / abs(ux) if abs(ux) > 1e-12 else 1e30, hy / abs(uy) if abs(uy) > 1e-12 else 1e30)
        cx, cy = s * ux + d * ux, s * uy + d * uy   # box boundary point, then d further out
        for tau in taus:
            for Rs in rss:
                if d < 7.0 * max(tau, 1.0) * Rs:
                    continue
                p = [Rs, 1.0, tau * Rs, cx, cy]
                fx, fy = oracle.alpha("TNFW", p, gx.ravel(), gy.ravel())
                ex, ey = oracle.alpha("TNFW", p, hx * tx, hy * ty)
                ix = interp(fx.reshape(N1, N1), tx, ty)
                iy = interp(fy.reshape(N1, N1), tx, ty)
                worst = max(worst, float(np.hypot(ix - ex, iy - ey).max() / np.hypot(ex, ey).max()))
    return worst


def test_interpolant_reproduces_polynomials_of_degree_seven():
    # the 8-point tensor interpolant is exact on x^a y^b with a, b <= 7 (a wrong node, weight or
    # index breaks this), and partition of unity holds at any point
    rng = np.random.default_rng(0)
    tx, ty = rng.uniform(-1, 1, 50), rng.uniform(-1, 1, 50)
    for a in range(8):
        for b in range(8):
            f = np.outer(NODES ** a, NODES ** b)
            np.testing.assert_allclose(interp(f, tx, ty), tx ** a * ty ** b, atol=1e-12)
    np.testing.assert_allclose(lagrange(tx).sum(axis=1), 1.0, atol=1e-13)
    # and not on degree 8
    f = np.outer(NODES ** 8, np.ones(N1))
    assert np.abs(interp(f, tx, ty) - tx ** 8).max() > 1e-4


@pytest.mark.parametrize("hx,hy", [(0.16, 0.08), (0.1, 0.1), (0.2, 0.05)])
@pytest.mark.parametrize("kappa", sorted(STATED))
def test_stated_far_field_bound_holds(kappa, hx, hy):
    err = worst_relative_error(kappa, hx, hy)
    assert err <= STATED[kappa], (kappa, hx, hy, err)


def test_bound_is_tight_and_the_cutoff_is_needed():
    # the stated numbers are close to the worst case (within 3x at kappa = 4), and kappa = 2,
    # which the API refuses, is an order of magnitude worse than kappa = 3
    e4 = worst_relative_error(4.0, 0.16, 0.08)
    assert e4 >= STATED[4.0] / 3.0, e4
    e2 = worst_relative_error(2.0, 0.16, 0.08)
    assert e2 >= 10.0 * STATED[3.0], e2

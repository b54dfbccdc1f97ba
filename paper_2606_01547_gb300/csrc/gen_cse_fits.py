"""Writes cse_fits.h: decompositions of the projected NFW and Hernquist profiles into cored
steep ellipsoids (CSEs), used by the NFW_ELLIPSE_CSE and HERNQUIST_ELLIPSE_CSE deflectors.

    kappa_hat(x) ~= sum_i a_i / (2 (sigma_i^2 + x^2)^(3/2)),   x = xi / Rs,

with kappa_hat_NFW(x) = 2 (1 - F(x)) / (x^2 - 1) and kappa_hat_Hernquist(x) =
((2 + x^2) F(x) - 3) / (x^2 - 1)^2 (F the NFW function).  The cores sigma_i are log-spaced; the
amplitudes a_i >= 0 minimise the relative error of kappa over log-spaced x by non-negative
least squares (Lawson & Hanson).  Positivity keeps the deflection sum free of cancellation.

Run by hand (needs numpy and scipy); the output is committed.  `python gen_cse_fits.py`.
"""
import os
import warnings

import numpy as np
from scipy import integrate
from scipy.optimize import nnls

N = 44
LOG_SIGMA = (-4.5, 4.5)
LOG_FIT = (-4.0, 4.0)
LOG_CHECK = (-3.0, 3.0)


def F(x):
    x = np.asarray(x, float)
    out = np.empty_like(x)
    lo, hi = x < 1, x > 1
    out[lo] = np.arccosh(1 / x[lo]) / np.sqrt(1 - x[lo] ** 2)
    out[hi] = np.arccos(1 / x[hi]) / np.sqrt(x[hi] ** 2 - 1)
    out[x == 1] = 1.0
    return out


def kappa_nfw(x):
    return 2 * (1 - F(x)) / (x * x - 1)


def kappa_hernquist(x):
    u = x * x - 1
    return ((2 + x * x) * F(x) - 3) / (u * u)


def basis(x, s):
    return 1 / (2 * (s[None, :] ** 2 + x[:, None] ** 2) ** 1.5)


def basis_alpha(x, s):
    # circular deflection of each CSE: (1/x)(1/s - 1/sqrt(s^2 + x^2))
    return (1 / x[:, None]) * (1 / s[None, :] - 1 / np.sqrt(s[None, :] ** 2 + x[:, None] ** 2))


def alpha_exact(kf, xs):
    # (2/x) int_0^x kappa(t) t dt by adaptive quadrature (x = 1 handled as an interior point)
    g = lambda t: kf(np.array([t]))[0] * t
    out = []
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        for x in xs:
            # log-spaced pieces resolve the logarithmic cusp at t = 0
            edges = np.concatenate([[0.0], np.logspace(-8, np.log10(x), 40)])
            v = sum(integrate.quad(g, a, b, limit=200, epsabs=0, epsrel=1e-13)[0] for a, b in zip(edges[:-1], edges[1:]))
            out.append(2 * v / x)
    return np.array(out)


def fit(kf):
    s = np.logspace(*LOG_SIGMA, N)
    x = np.logspace(*LOG_FIT, 4000)
    x = x[np.abs(x - 1) > 1e-3]
    k = kf(x)
    a, _ = nnls(basis(x, s) / k[:, None], np.ones_like(k), maxiter=200000)
    xt = np.logspace(*LOG_CHECK, 3001)
    xt = xt[np.abs(xt - 1) > 1e-3]
    ek = np.abs(basis(xt, s) @ a / kf(xt) - 1).max()
    xa = np.logspace(*LOG_CHECK, 121)
    xa = xa[np.abs(xa - 1) > 1e-3]
    ea = np.abs(basis_alpha(xa, s) @ a / alpha_exact(kf, xa) - 1).max()
    return s, a, ek, ea


def main():
    lines = ["// Generated by gen_cse_fits.py; do not edit.  Cored-steep-ellipsoid decompositions",
             "//   kappa_hat(x) ~= sum_i a_i / (2 (sigma_i^2 + x^2)^(3/2)),  x = xi / Rs,",
             f"// with {N} log-spaced cores sigma_i in [1e{LOG_SIGMA[0]}, 1e{LOG_SIGMA[1]}] and amplitudes a_i >= 0",
             f"// fitted by non-negative least squares to the relative error of kappa at 4000 log-spaced",
             f"// x in [1e{LOG_FIT[0]}, 1e{LOG_FIT[1]}].",
             "#pragma once", "", "namespace ls {", "", f"constexpr int kCseTerms = {N};", ""]
    for name, kf in (("Nfw", kappa_nfw), ("Hernquist", kappa_hernquist)):
        s, a, ek, ea = fit(kf)
        lines.append(f"// {name}: max relative error on x in [1e{LOG_CHECK[0]}, 1e{LOG_CHECK[1]}]: "
                     f"kappa {ek:.2e}, circular deflection {ea:.2e}.")
        lines.append(f"static __constant__ float kCse{name}Sigma[kCseTerms] = {{")
        lines += ["    " + ", ".join(f"{v:.9e}f" for v in s[i:i + 4]) + "," for i in range(0, N, 4)]
        lines.append("};")
        lines.append(f"static __constant__ float kCse{name}Amp[kCseTerms] = {{")
        lines += ["    " + ", ".join(f"{v:.9e}f" for v in a[i:i + 4]) + "," for i in range(0, N, 4)]
        lines.append("};")
        lines.append("")
        print(name, "kappa", ek, "alpha", ea, "nonzero", np.count_nonzero(a))
    lines += ["}  // namespace ls", ""]
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cse_fits.h")
    with open(out, "w") as f:
        f.write("\n".join(lines))
    print("wrote", out)


if __name__ == "__main__":
    main()

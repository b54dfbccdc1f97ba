"""Write nfw_tnfw_mass.txt: 40-digit projected masses of the NFW and truncated-NFW
(n = 1 truncation, tau = 5) densities, by mpmath quadrature of the 3-D density.

m(x) = int_0^inf r^2 rho(r) g(r, x) dr with g = 1 for r <= x and 1 - sqrt(1 - x^2/r^2)
beyond (the fraction of a spherical shell inside the cylinder of radius x);
rho = 1/(r (1+r)^2) for NFW, times tau^2/(tau^2 + r^2) for the truncated profile
(Baltz, Marshall & Oguri 2009).  No oracle code is involved.
"""
import os

import mpmath as mp

mp.mp.dps = 40
XS = ["1e-4", "1e-3", "0.01", "0.1", "0.5", "0.9", "0.999", "1", "1.001", "1.5", "3", "10", "100", "1000"]


def m_of_x(x, tau=None):
    rho = (lambda r: 1 / (r * (1 + r) ** 2)) if tau is None else \
        (lambda r: tau * tau / (r * (1 + r) ** 2 * (tau * tau + r * r)))
    inner = mp.quad(lambda r: r * r * rho(r), [0, x])
    outer = mp.quad(lambda r: r * r * rho(r) * (x * x / (r * r)) / (1 + mp.sqrt(1 - x * x / (r * r))),
                    [x, 2 * x, 10 * x, 100 * x, mp.inf])
    return inner + outer


if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "nfw_tnfw_mass.txt")
    with open(out, "w") as fh:
        fh.write("# x  m_NFW(x)  m_TNFW(x; tau=5)   (mpmath, 40 digits; see make_golden.py)\n")
        for xs in XS:
            x = mp.mpf(xs)
            fh.write(f"{xs} {mp.nstr(m_of_x(x), 25)} {mp.nstr(m_of_x(x, mp.mpf(5)), 25)}\n")

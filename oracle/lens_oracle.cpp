// Plain FP64 CPU oracle for the lensed-image simulation path.
//
// TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct definition
// that the CUDA path is checked against.  Only the test-suite, the smoke check and
// the CPU-baseline leg of the benchmark may load it; the product library never
// does, and it shares no code (no headers, helpers or tables) with the CUDA path.
//
// What the paper fixes: the three steps of image simulation (ray-trace an
// observer-plane grid through the deflectors, evaluate the source surface
// brightness on the traced coordinates, convolve with the PSF; section
// "Improvements over lenstronomy in image simulation"), and the profile names
// (deflection table: EPL, NIE/SIE, SHEAR, SIS, NFW, TNFW; light table:
// SERSIC_ELLIPSE, SERSIC_ELLIPSE_Q_PHI).  The paper prints no formula, so each
// profile below follows its standard published definition, named beside it,
// and each reading the paper leaves open is marked "reading:".
//
// Everything is templated on the scalar type T, instantiated for double and for
// a forward-mode dual number, so the likelihood gradient is the exact derivative
// of the same definition (used for the gradient-based fitting the paper adds via
// automatic differentiation, section "Improvements over lenstronomy in lens
// modelling").
//
// Build: g++ -O2 -std=c++17 -fopenmp -fPIC -shared (no fast-math).

#include <cmath>
#include <cstdio>
#include <cstring>
#include <cstdint>
#include <vector>
#include <algorithm>
#include <type_traits>
#ifdef _OPENMP
#include <omp.h>
#endif

// System description passed in by the Python wrapper (plain C layout).
typedef struct {
  int nx, ny, s;
  double dpix, x0, y0;
  int n_defl;
  const int* defl_type;     // [n_defl]
  const double* defl_p;     // [n_defl][kDeflParams]
  int n_sub;
  const double* sub;        // SoA [5][n_sub]: cx, cy, Rs, alpha_Rs, r_t (TNFW)
  int src_type;
  double src_p[8];
  int k;                    // PSF size (odd); 0 = no PSF
  const double* psf;        // [k][k]
  const double* src_coef;   // SHAPELETS amplitudes (n_src_coef of them), else unused
  int n_src_coef;
} oracle_system;

// Parameters per deflector in defl_p (the widest layout, EPL_MULTIPOLE_M1M3M4, has 12).
constexpr int kDeflParams = 12;

namespace {

// ---------------------------------------------------------------------------
// Forward-mode dual number with N tangent directions.
// ---------------------------------------------------------------------------
template <int N>
struct Dual {
  double v;
  double d[N];
  Dual() : v(0.0) { for (int i = 0; i < N; ++i) d[i] = 0.0; }
  Dual(double x) : v(x) { for (int i = 0; i < N; ++i) d[i] = 0.0; }
};

template <int N> inline Dual<N> chain(const Dual<N>& a, double val, double dval) {
  Dual<N> r(val);
  for (int i = 0; i < N; ++i) r.d[i] = dval * a.d[i];
  return r;
}
template <int N> inline Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r(a.v + b.v); for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i]; return r; }
template <int N> inline Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r(a.v - b.v); for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i]; return r; }
template <int N> inline Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r(a.v * b.v); for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r; }
template <int N> inline Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r(a.v / b.v);
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v);
  return r; }
template <int N> inline Dual<N> operator-(const Dual<N>& a) {
  Dual<N> r(-a.v); for (int i = 0; i < N; ++i) r.d[i] = -a.d[i]; return r; }
template <int N> inline Dual<N> operator+(const Dual<N>& a, double b) { Dual<N> r = a; r.v += b; return r; }
template <int N> inline Dual<N> operator+(double b, const Dual<N>& a) { Dual<N> r = a; r.v += b; return r; }
template <int N> inline Dual<N> operator-(const Dual<N>& a, double b) { Dual<N> r = a; r.v -= b; return r; }
template <int N> inline Dual<N> operator-(double b, const Dual<N>& a) { return (-a) + b; }
template <int N> inline Dual<N> operator*(const Dual<N>& a, double b) {
  Dual<N> r(a.v * b); for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b; return r; }
template <int N> inline Dual<N> operator*(double b, const Dual<N>& a) { return a * b; }
template <int N> inline Dual<N> operator/(const Dual<N>& a, double b) { return a * (1.0 / b); }
template <int N> inline Dual<N> operator/(double a, const Dual<N>& b) {
  Dual<N> r(a / b.v); for (int i = 0; i < N; ++i) r.d[i] = -a * b.d[i] / (b.v * b.v); return r; }
template <int N> inline Dual<N>& operator+=(Dual<N>& a, const Dual<N>& b) { a = a + b; return a; }
template <int N> inline Dual<N>& operator-=(Dual<N>& a, const Dual<N>& b) { a = a - b; return a; }

template <int N> inline Dual<N> sqrt(const Dual<N>& a) { double s = std::sqrt(a.v); return chain(a, s, 0.5 / s); }
template <int N> inline Dual<N> exp(const Dual<N>& a) { double e = std::exp(a.v); return chain(a, e, e); }
template <int N> inline Dual<N> log(const Dual<N>& a) { return chain(a, std::log(a.v), 1.0 / a.v); }
template <int N> inline Dual<N> sin(const Dual<N>& a) { return chain(a, std::sin(a.v), std::cos(a.v)); }
template <int N> inline Dual<N> cos(const Dual<N>& a) { return chain(a, std::cos(a.v), -std::sin(a.v)); }
template <int N> inline Dual<N> atan(const Dual<N>& a) { return chain(a, std::atan(a.v), 1.0 / (1.0 + a.v * a.v)); }
template <int N> inline Dual<N> atanh(const Dual<N>& a) { return chain(a, std::atanh(a.v), 1.0 / (1.0 - a.v * a.v)); }
template <int N> inline Dual<N> atan2(const Dual<N>& y, const Dual<N>& x) {
  double den = x.v * x.v + y.v * y.v;
  Dual<N> r(std::atan2(y.v, x.v));
  for (int i = 0; i < N; ++i) r.d[i] = (x.v * y.d[i] - y.v * x.d[i]) / den;
  return r;
}

inline double val(double x) { return x; }
template <int N> inline double val(const Dual<N>& x) { return x.v; }

using std::sqrt; using std::exp; using std::log; using std::sin; using std::cos;
using std::atan; using std::atanh; using std::atan2;

constexpr double kPi = 3.14159265358979323846;
constexpr double kLn2 = 0.69314718055994530942;

// Profile type codes of this oracle's C interface (its own numbering).
enum { O_SIS = 0, O_SIE = 1, O_EPL = 2, O_SHEAR = 3, O_POINT_MASS = 4, O_NFW = 5,
       O_TNFW = 6, O_EPL_E1E2 = 7, O_SIE_E1E2 = 8, O_MULTIPOLE = 9, O_EPL_MULTIPOLE_M1M3M4 = 10,
       O_CSE = 11, O_NFW_ELLIPSE_CSE = 12, O_HERNQUIST_ELLIPSE_CSE = 13, O_MULTIPOLE_ELL = 14 };
enum { O_SERSIC_ELLIPSE_Q_PHI = 0, O_SERSIC_ELLIPSE = 1, O_SERSIC = 2, O_SHAPELETS = 3 };

// ---------------------------------------------------------------------------
// Ellipticity helpers.
// reading: the paper does not state the e1/e2 convention; the lenstronomy one is
// used: phi = atan2(e2, e1)/2, c = sqrt(e1^2+e2^2), q = (1-c)/(1+c).
// reading: the ellipse frame is x' = cos(phi) dx + sin(phi) dy,
//          y' = -sin(phi) dx + cos(phi) dy (phi from +x toward +y).
// ---------------------------------------------------------------------------
template <class T> inline void e1e2_to_qphi(const T& e1, const T& e2, T& q, T& phi) {
  phi = 0.5 * atan2(e2, e1);
  T c = sqrt(e1 * e1 + e2 * e2);
  q = (1.0 - c) / (1.0 + c);
}

// ---------------------------------------------------------------------------
// Deflection profiles.  Each returns the deflection vector (ax, ay) in arcsec.
// ---------------------------------------------------------------------------

// SIS (deflection table row SIS): alpha = theta_E * (dx, dy) / r.
// reading: alpha = 0 when r < 1e-12 arcsec.
template <class T>
void alpha_sis(const T& x, const T& y, const T& thetaE, const T& cx, const T& cy, T& ax, T& ay) {
  T dx = x - cx, dy = y - cy;
  T r = sqrt(dx * dx + dy * dy);
  if (val(r) < 1e-12) { ax = 0.0; ay = 0.0; return; }
  ax = thetaE * dx / r;
  ay = thetaE * dy / r;
}

// Point mass: alpha = theta_E^2 (dx, dy) / r^2 (test profile only).
template <class T>
void alpha_point_mass(const T& x, const T& y, const T& thetaE, const T& cx, const T& cy, T& ax, T& ay) {
  T dx = x - cx, dy = y - cy;
  T r2 = dx * dx + dy * dy;
  if (val(r2) < 1e-24) { ax = 0.0; ay = 0.0; return; }
  ax = thetaE * thetaE * dx / r2;
  ay = thetaE * thetaE * dy / r2;
}

// SIE (deflection table row NIE/SIE), Kormann, Schneider & Bartelmann (1994) in the
// form kappa = b / (2 psi), psi = sqrt(q^2 x'^2 + y'^2), b = theta_E sqrt(q), so that
// kappa = theta_E / (2 sqrt(q x'^2 + y'^2 / q)).  In the ellipse frame
//   a'_x = b/sqrt(1-q^2) atan (sqrt(1-q^2) x'/psi),
//   a'_y = b/sqrt(1-q^2) atanh(sqrt(1-q^2) y'/psi).
// reading: |1-q| < 1e-6 takes the SIS limit.
template <class T>
void alpha_sie(const T& x, const T& y, const T& thetaE, const T& q, const T& phi,
               const T& cx, const T& cy, T& ax, T& ay) {
  T c = cos(phi), s = sin(phi);
  T dx = x - cx, dy = y - cy;
  T xp = c * dx + s * dy, yp = -s * dx + c * dy;
  T r2 = dx * dx + dy * dy;
  if (std::sqrt(val(r2)) < 1e-12) { ax = 0.0; ay = 0.0; return; }
  T apx, apy;
  if (std::fabs(1.0 - val(q)) < 1e-6) {
    T r = sqrt(r2);
    apx = thetaE * xp / r;
    apy = thetaE * yp / r;
  } else {
    T b = thetaE * sqrt(q);
    T psi = sqrt(q * q * xp * xp + yp * yp);
    T e = sqrt(1.0 - q * q);
    apx = b / e * atan(e * xp / psi);
    apy = b / e * atanh(e * yp / psi);
  }
  ax = c * apx - s * apy;
  ay = s * apx + c * apy;
}

// EPL (deflection table row EPL), Tessore & Metcalf (2015).  With t = gamma - 1,
// elliptical radius R = sqrt(q^2 x'^2 + y'^2), e^{i phi_e} = (q x' + i y') / R and
// b = theta_E sqrt(q), so that kappa = (3-gamma)/2 (theta_E / sqrt(q x'^2 + y'^2/q))^(gamma-1):
//   a' = 2b/(1+q) (b/R)^(t-1) Omega,   Omega = sum_n Omega_n,
//   Omega_0 = e^{i phi_e},
//   Omega_n = -f (2n-2+t)/(2n+2-t) e^{2 i phi_e} Omega_{n-1},   f = (1-q)/(1+q),
// i.e. e^{i phi_e} 2F1(1, t/2; 2-t/2; -f e^{2 i phi_e}).  The series is summed until a
// term is below 1e-17 of the running sum (at most 400 terms).
template <class T>
void alpha_epl(const T& x, const T& y, const T& thetaE, const T& gamma, const T& q, const T& phi,
               const T& cx, const T& cy, T& ax, T& ay) {
  T c = cos(phi), s = sin(phi);
  T dx = x - cx, dy = y - cy;
  T xp = c * dx + s * dy, yp = -s * dx + c * dy;
  T R = sqrt(q * q * xp * xp + yp * yp);
  if (val(R) < 1e-12) { ax = 0.0; ay = 0.0; return; }
  T t = gamma - 1.0;
  T b = thetaE * sqrt(q);
  T er = q * xp / R, ei = yp / R;
  T f = (1.0 - q) / (1.0 + q);
  T zr = -f * (er * er - ei * ei), zi = -f * (2.0 * er * ei);
  T om_r = er, om_i = ei;
  T sr = om_r, si = om_i;
  for (int n = 1; n <= 400; ++n) {
    T coef = (2.0 * n - 2.0 + t) / (2.0 * n + 2.0 - t);
    T nr = coef * (om_r * zr - om_i * zi);
    T ni = coef * (om_r * zi + om_i * zr);
    om_r = nr; om_i = ni;
    sr += om_r; si += om_i;
    double mag = std::hypot(val(om_r), val(om_i));
    double tot = std::hypot(val(sr), val(si));
    if (mag <= 1e-17 * tot) break;
  }
  T pref = 2.0 * b / (1.0 + q) * exp((t - 1.0) * log(b / R));
  T apx = pref * sr, apy = pref * si;
  ax = c * apx - s * apy;
  ay = s * apx + c * apy;
}

// External shear (deflection table row SHEAR): alpha = (g1 x + g2 y, g2 x - g1 y)
// about the origin.
template <class T>
void alpha_shear(const T& x, const T& y, const T& g1, const T& g2, T& ax, T& ay) {
  ax = g1 * x + g2 * y;
  ay = g2 * x - g1 * y;
}

// NFW helper F(x) (Bartelmann 1996; Wright & Brainerd 2000):
//   F = atanh(sqrt(1-x^2))/sqrt(1-x^2) for x<1, 1 at x=1, atan(sqrt(x^2-1))/sqrt(x^2-1) for x>1,
// i.e. sum_k (-v)^k/(2k+1) with v = x^2-1; that series is used for |v| < 1e-4.
// For x < 1 the arccosh is evaluated as ln((1 + u)/x) with u = sqrt((1-x)(1+x)), which
// is the same function; the atanh(u) route loses ~1e-10 absolutely near u -> 1 and the
// ln(x/2) + F(x) cancellation of the NFW/TNFW masses at small x amplifies that.
template <class T> T nfw_F(const T& x) {
  T v = x * x - 1.0;
  if (std::fabs(val(v)) < 1e-4) {
    T term = T(1.0), sum = T(1.0);
    for (int k = 1; k <= 8; ++k) { term = term * (-v); sum += term / (2.0 * k + 1.0); }
    return sum;
  }
  if (val(v) > 0.0) { T u = sqrt(v); return atan(u) / u; }
  T u = sqrt((1.0 - x) * (1.0 + x));
  return log((1.0 + u) / x) / u;
}

// Normalisation shared by NFW and TNFW.  reading: alpha_Rs is the deflection of the
// untruncated NFW at r = Rs (lenstronomy's convention), so 4 kappa_s Rs = alpha_Rs / (1 - ln 2).
// The radial deflection is 4 kappa_s Rs M(x)/x with x = r/Rs, hence the vector
// alpha = alpha_Rs / ((1 - ln 2) Rs) * M(x)/x^2 * (dx, dy).
// reading: x is floored at 1e-6 (alpha -> 0 continuously at the centre).

// NFW: M(x) = h(x) = ln(x/2) + F(x).
template <class T>
void alpha_nfw(const T& x, const T& y, const T& Rs, const T& alphaRs, const T& cx, const T& cy,
               T& ax, T& ay) {
  T dx = x - cx, dy = y - cy;
  T r = sqrt(dx * dx + dy * dy);
  T xx = r / Rs;
  if (val(xx) < 1e-6) xx = T(1e-6);
  T h = log(xx / 2.0) + nfw_F(xx);
  T k = alphaRs / ((1.0 - kLn2) * Rs) * h / (xx * xx);
  ax = k * dx;
  ay = k * dy;
}

// Truncated NFW (deflection table row TNFW), Baltz, Marshall & Oguri (2009), n = 1
// truncation: rho ~ [x (1+x)^2]^-1 * tau^2 / (tau^2 + x^2), tau = r_t / Rs.
//   M(x) = tau^2/(tau^2+1)^2 [ (tau^2 + 1 + 2(x^2-1)) F(x) + tau pi + (tau^2-1) ln tau
//          + sqrt(tau^2+x^2) (-pi + L(x) (tau^2-1)/tau) ],
//   L(x) = ln( x / (sqrt(tau^2+x^2) + tau) ).
template <class T>
T tnfw_M(const T& xx, const T& tau) {
  T t2 = tau * tau;
  T S = sqrt(t2 + xx * xx);
  T L = log(xx / (S + tau));
  T F = nfw_F(xx);
  T br = (t2 + 1.0 + 2.0 * (xx * xx - 1.0)) * F + tau * kPi + (t2 - 1.0) * log(tau)
         + S * (-kPi + L * (t2 - 1.0) / tau);
  return t2 / ((t2 + 1.0) * (t2 + 1.0)) * br;
}

template <class T>
void alpha_tnfw(const T& x, const T& y, const T& Rs, const T& alphaRs, const T& rt,
                const T& cx, const T& cy, T& ax, T& ay) {
  T dx = x - cx, dy = y - cy;
  T r = sqrt(dx * dx + dy * dy);
  T xx = r / Rs;
  if (val(xx) < 1e-6) xx = T(1e-6);
  T tau = rt / Rs;
  T M = tnfw_M(xx, tau);
  T k = alphaRs / ((1.0 - kLn2) * Rs) * M / (xx * xx);
  ax = k * dx;
  ay = k * dy;
}

// Circular multipole of order m (deflection table rows MULTIPOLE and EPL_MULTIPOLE_M1M3M4;
// the m-th angular Fourier mode of the convergence about a centre, as in Chu et al. 2013):
//   kappa = r_E a_m cos(m (phi - phi_m)) / (2 r),
// whose potential is psi = r_E a_m r cos(m dphi) / (1 - m^2) for m >= 2 and
// psi = (r_E a_1 / 2) r ln(r / r_E) cos(dphi) for m = 1 (dphi = phi - phi_m); alpha = grad psi,
// written as the radial and tangential derivatives rotated back to (x, y).
// reading: parameters m, a_m, phi_m, cx, cy, r_E; a_m is dimensionless, relative to the
// isothermal convergence r_E / (2 r); alpha = 0 when r < 1e-12 arcsec.
template <class T>
void alpha_multipole(const T& x, const T& y, int m, const T& am, const T& phim, const T& cx, const T& cy,
                     const T& rE, T& ax, T& ay) {
  T dx = x - cx, dy = y - cy;
  T r = sqrt(dx * dx + dy * dy);
  if (val(r) < 1e-12) { ax = T(0.0); ay = T(0.0); return; }
  T phi = atan2(dy, dx);
  T d = phi - phim;
  T ar, at;  // d psi / d r and (1/r) d psi / d phi
  if (m == 1) {
    T B = 0.5 * rE * am;
    T L = log(r / rE);
    ar = B * (L + 1.0) * cos(d);
    at = -B * L * sin(d);
  } else {
    T A = rE * am / (1.0 - (double)m * m);
    ar = A * cos((double)m * d);
    at = -A * (double)m * sin((double)m * d);
  }
  T c = cos(phi), sn = sin(phi);
  ax = ar * c - at * sn;
  ay = ar * sn + at * c;
}

// Adaptive Gauss-Kronrod (7/15 points) on [a, b] to an absolute tolerance, for smooth
// integrands; plain recursion.  An interval is also accepted once the Gauss-Kronrod difference
// is at the rounding level of its own sum (50 eps sum |w f|), and recursion stops at depth 20.
template <class F>
double gk15(const F& f, double a, double b, double tol, int depth = 0) {
  static const double xk[8] = {0.991455371120812639206854697526329, 0.949107912342758524526189684047851,
                               0.864864423359769072789712788640926, 0.741531185599394439863864773280788,
                               0.586087235467691130294144845693013, 0.405845151377397166906606412076961,
                               0.207784955007898467600689403773245, 0.0};
  static const double wk[8] = {0.022935322010529224963732008058970, 0.063092092629978553290700663189204,
                               0.104790010322250183839876322541518, 0.140653259715525918745189590510238,
                               0.169004726639267902826583426598550, 0.190350578064785409913256402421014,
                               0.204432940075298892414161999234649, 0.209482141084727828012999174891714};
  static const double wg[4] = {0.129484966168869693270611432679082, 0.279705391489276667901467771423780,
                               0.381830050505118944950369775488975, 0.417959183673469387755102040816327};
  const double c = 0.5 * (a + b), h = 0.5 * (b - a);
  double fc = f(c);
  double K = wk[7] * fc, G = wg[3] * fc, Kabs = wk[7] * std::fabs(fc);
  for (int j = 0; j < 7; ++j) {
    const double f1 = f(c - h * xk[j]), f2 = f(c + h * xk[j]);
    K += wk[j] * (f1 + f2);
    Kabs += wk[j] * (std::fabs(f1) + std::fabs(f2));
    if (j & 1) G += wg[j / 2] * (f1 + f2);
  }
  K *= h; G *= h; Kabs *= std::fabs(h);
  const double err = std::fabs(K - G);
  if (!(err == err) || err <= tol || err <= 50.0 * 2.220446049250313e-16 * Kabs || depth >= 20) return K;
  return gk15(f, a, c, 0.5 * tol, depth + 1) + gk15(f, c, b, 0.5 * tol, depth + 1);
}

// Deflection of an elliptical convergence kappa(xi_c^2), xi_c^2 = x'^2 + y'^2/q^2, in its frame,
// by the Schramm (1990) integrals
//   alpha'_x = q x' J_0,  alpha'_y = q y' J_1,
//   J_n = int_0^1 kappa(xi(u)^2) / (1 - (1 - q^2) u)^(n + 1/2) du,  xi(u)^2 = u (x'^2 + y'^2 / (1 - (1-q^2) u)),
// with u = t^2 so that a logarithmic central cusp leaves a smooth integrand; adaptive quadrature
// to the absolute tolerance `tol` (FP64 only; not part of the differentiated model).
template <class K>
void schramm_alpha(const K& kappa, double xp, double yp, double q, double tol, double& axp, double& ayp) {
  const double e = 1.0 - q * q;
  auto xi2 = [&](double u) { return u * (xp * xp + yp * yp / (1.0 - e * u)); };
  const double J0 = gk15([&](double t) { const double u = t * t; return 2.0 * t * kappa(xi2(u)) / std::sqrt(1.0 - e * u); },
                         0.0, 1.0, tol);
  const double J1 = gk15([&](double t) { const double u = t * t; return 2.0 * t * kappa(xi2(u)) / std::pow(1.0 - e * u, 1.5); },
                         0.0, 1.0, tol);
  axp = q * xp * J0;
  ayp = q * yp * J1;
}

// Elliptical-convergence profile: the frame of (q, phi, cx, cy), then the Schramm integrals.
template <class K>
void alpha_elliptical(const K& kappa, double x, double y, double q, double phi, double cx, double cy, double tol,
                      double& ax, double& ay) {
  const double c = std::cos(phi), sn = std::sin(phi);
  const double dx = x - cx, dy = y - cy;
  const double xp = c * dx + sn * dy, yp = -sn * dx + c * dy;
  double axp, ayp;
  schramm_alpha(kappa, xp, yp, q, tol, axp, ayp);
  ax = c * axp - sn * ayp;
  ay = sn * axp + c * ayp;
}

// Cored steep ellipsoid (deflection table row CSE; Oguri 2021):
//   kappa = A / (2 (s^2 + xi_c^2)^(3/2)).
// reading: parameters A, s, e1, e2, cx, cy with the e1/e2 convention of the other profiles.
inline void alpha_cse(double x, double y, double A, double s, double q, double phi, double cx, double cy,
                      double& ax, double& ay) {
  auto kap = [&](double xi2) { return A / (2.0 * std::pow(s * s + xi2, 1.5)); };
  alpha_elliptical(kap, x, y, q, phi, cx, cy, 1e-15 * (std::fabs(A) / (s * s * s) + 1e-300), ax, ay);
}

// Projected NFW and Hernquist convergences in units of their normalisation, x = xi / Rs
// (Bartelmann 1996; Hernquist 1990), with F(x) the NFW function:
//   kappa_NFW = 2 (1 - F(x)) / (x^2 - 1),   kappa_Hernquist = ((2 + x^2) F(x) - 3) / (x^2 - 1)^2;
// for |v| < 0.1, v = x^2 - 1, both use their series in v (F = sum (-v)^k / (2k+1)), which
// removes the cancellation of the closed forms there (30 terms: below 1e-30 truncation).
inline double kappa_hat_nfw(double x) {
  const double v = x * x - 1.0;
  if (std::fabs(v) < 0.1) {
    double s = 0.0, pw = 1.0;  // (1 - F)/v = sum_{k>=1} (-1)^(k+1) v^(k-1) / (2k+1)
    for (int k = 1; k <= 30; ++k) { s += ((k & 1) ? 1.0 : -1.0) * pw / (2.0 * k + 1.0); pw *= v; }
    return 2.0 * s;
  }
  return 2.0 * (1.0 - nfw_F<double>(x)) / v;
}
inline double kappa_hat_hernquist(double x) {
  const double v = x * x - 1.0;
  if (std::fabs(v) < 0.1) {
    double s = 0.0, pw = 1.0;  // bracket / v^2 = sum_{n>=2} (-1)^n 4 (n-1) / (4n^2 - 1) v^(n-2)
    for (int n = 2; n <= 32; ++n) { s += ((n & 1) ? -1.0 : 1.0) * 4.0 * (n - 1) / (4.0 * n * n - 1.0) * pw; pw *= v; }
    return s;
  }
  return ((2.0 + x * x) * nfw_F<double>(x) - 3.0) / (v * v);
}

// Elliptical NFW and Hernquist convergences (deflection table rows NFW_ELLIPSE_CSE and
// HERNQUIST_ELLIPSE_CSE; the oracle takes the exact profiles, not a CSE decomposition).
// reading: xi^2 = q x'^2 + y'^2/q (area-preserving, as for SIE and the Sersic source);
// NFW: Rs, alpha_Rs, e1, e2, cx, cy with kappa = kappa_s kappa_hat_NFW(xi/Rs),
// kappa_s Rs = alpha_Rs / (4 (1 - ln 2)); Hernquist: sigma0, Rs, e1, e2, cx, cy with
// kappa = sigma0 kappa_hat_Hernquist(xi/Rs).
inline void alpha_nfw_ellipse(double x, double y, double Rs, double alphaRs, double q, double phi, double cx,
                              double cy, double& ax, double& ay) {
  const double ks = alphaRs / (4.0 * (1.0 - kLn2) * Rs);
  auto kap = [&](double xi2c) { return ks * kappa_hat_nfw(std::max(std::sqrt(q * xi2c), 1e-300) / Rs); };
  alpha_elliptical(kap, x, y, q, phi, cx, cy, 1e-15 * std::fabs(ks), ax, ay);
}
inline void alpha_hernquist_ellipse(double x, double y, double sigma0, double Rs, double q, double phi, double cx,
                                    double cy, double& ax, double& ay) {
  auto kap = [&](double xi2c) { return sigma0 * kappa_hat_hernquist(std::max(std::sqrt(q * xi2c), 1e-300) / Rs); };
  alpha_elliptical(kap, x, y, q, phi, cx, cy, 1e-15 * std::fabs(sigma0), ax, ay);
}

// Elliptical multipole of order m (deflection table row MULTIPOLE_ELL).
// reading: in the frame of an ellipse of axis ratio q and position angle phi_e about (cx, cy),
//   kappa = r_E a_m cos(m (varphi - phi_m')) / (2 R),  R^2 = q x''^2 + y''^2 / q,
// varphi = atan2(y'' / sqrt(q), x'' sqrt(q)) the elliptical angle, phi_m' = phi_m - phi_e;
// parameters m, a_m, phi_m, q, phi_e, cx, cy, r_E.  q = 1 is the circular multipole above.
// kappa r depends on the polar angle theta alone: with h(theta) = 2 kappa r and its Fourier
// coefficients c_k, the potential is psi = r F(theta) + (1/2) r ln(r / r_E) h_1(theta), where
// F = sum_{k != +-1} c_k e^{i k theta} / (1 - k^2) solves F + F'' = h - h_1 and the k = +-1 part
// h_1 (present for odd m) is carried by the r ln r term, whose Laplacian is h_1 / r; so
// laplacian(psi) = h / r = 2 kappa.  alpha = grad psi.  The c_k come from the trapezoid rule on
// kEllN points, which converges geometrically for this analytic periodic h (its singularities
// lie at |Im theta| = atanh(q)); kept up to order m + 256 (q >= 0.2).
constexpr int kEllN = 4096;
struct EllCoef {
  int m = -1;
  double q = -1.0, dphi = 0.0;
  int K = 0;
  std::vector<double> re, im;  // c_k / (a_m r_E), k = 0..K
};

inline const EllCoef& ell_coefficients(int m, double q, double dphi) {
  static thread_local EllCoef c;
  if (c.m == m && c.q == q && c.dphi == dphi) return c;
  c.m = m;
  c.q = q;
  c.dphi = dphi;
  c.K = std::min(m + 256, kEllN / 4);
  std::vector<double> h(kEllN), cs(kEllN), sn(kEllN);
  const double sq = std::sqrt(q);
  for (int j = 0; j < kEllN; ++j) {
    const double th = 2.0 * kPi * j / kEllN;
    cs[j] = std::cos(th);
    sn[j] = std::sin(th);
    const double g = std::sqrt(q * cs[j] * cs[j] + sn[j] * sn[j] / q);  // R / r
    const double vphi = std::atan2(sn[j] / sq, sq * cs[j]);
    h[j] = std::cos(m * (vphi - dphi)) / g;                             // 2 kappa r / (a_m r_E)
  }
  c.re.assign(c.K + 1, 0.0);
  c.im.assign(c.K + 1, 0.0);
  for (int k = 0; k <= c.K; ++k) {
    double sr = 0.0, si = 0.0;
    for (int j = 0; j < kEllN; ++j) {
      const int idx = (int)(((long long)k * j) % kEllN);
      sr += h[j] * cs[idx];
      si -= h[j] * sn[idx];
    }
    c.re[k] = sr / kEllN;
    c.im[k] = si / kEllN;
  }
  return c;
}

inline void alpha_multipole_ell(double x, double y, int m, double am, double phim, double q, double phie,
                                double cx, double cy, double rE, double& ax, double& ay) {
  const double ce = std::cos(phie), se = std::sin(phie);
  const double dx = x - cx, dy = y - cy;
  const double xp = ce * dx + se * dy, yp = -se * dx + ce * dy;
  const double r = std::sqrt(xp * xp + yp * yp);
  if (r < 1e-12) { ax = 0.0; ay = 0.0; return; }
  const EllCoef& c = ell_coefficients(m, q, phim - phie);
  const double s = am * rE;
  const double cth = xp / r, sth = yp / r;
  // F and F' from the harmonics k = 0 and 2..K (h real: c_{-k} = conj(c_k))
  double F = c.re[0], Fd = 0.0;
  double zr = cth, zi = sth;  // e^{i k theta}, k = 1
  for (int k = 2; k <= c.K; ++k) {
    const double nr = zr * cth - zi * sth, ni = zr * sth + zi * cth;
    zr = nr;
    zi = ni;
    const double w = 2.0 / (1.0 - (double)k * k);
    const double pr = c.re[k] * zr - c.im[k] * zi;  // Re(c_k e^{ik theta})
    const double pi = c.re[k] * zi + c.im[k] * zr;  // Im(c_k e^{ik theta})
    F += w * pr;
    Fd -= w * k * pi;
  }
  // the resonant part h_1 = A cos(theta) + B sin(theta)
  const double A = 2.0 * c.re[1], B = -2.0 * c.im[1];
  const double h1 = A * cth + B * sth, h1d = -A * sth + B * cth;
  const double L = std::log(r / rE);
  const double ar = s * (F + 0.5 * (L + 1.0) * h1);
  const double at = s * (Fd + 0.5 * L * h1d);
  const double axp = ar * cth - at * sth, ayp = ar * sth + at * cth;
  ax = ce * axp - se * ayp;
  ay = se * axp + ce * ayp;
}

// Dispatch one profile; p holds the profile's parameters in the order of its layout.
template <class T>
int alpha_profile(int type, const T* p, const T& x, const T& y, T& ax, T& ay) {
  switch (type) {
    case O_SIS: alpha_sis(x, y, p[0], p[1], p[2], ax, ay); return 0;
    case O_SIE: alpha_sie(x, y, p[0], p[1], p[2], p[3], p[4], ax, ay); return 0;
    case O_EPL: alpha_epl(x, y, p[0], p[1], p[2], p[3], p[4], p[5], ax, ay); return 0;
    case O_SHEAR: alpha_shear(x, y, p[0], p[1], ax, ay); return 0;
    case O_POINT_MASS: alpha_point_mass(x, y, p[0], p[1], p[2], ax, ay); return 0;
    case O_NFW: alpha_nfw(x, y, p[0], p[1], p[2], p[3], ax, ay); return 0;
    case O_TNFW: alpha_tnfw(x, y, p[0], p[1], p[2], p[3], p[4], ax, ay); return 0;
    case O_EPL_E1E2: {
      T q, phi; e1e2_to_qphi(p[2], p[3], q, phi);
      alpha_epl(x, y, p[0], p[1], q, phi, p[4], p[5], ax, ay); return 0;
    }
    case O_SIE_E1E2: {
      T q, phi; e1e2_to_qphi(p[1], p[2], q, phi);
      alpha_sie(x, y, p[0], q, phi, p[3], p[4], ax, ay); return 0;
    }
    case O_MULTIPOLE: {
      const int m = (int)std::lround(val(p[0]));
      if (m < 1 || std::fabs(val(p[0]) - m) > 1e-6 || !(val(p[5]) > 0.0)) return -1;
      alpha_multipole(x, y, m, p[1], p[2], p[3], p[4], p[5], ax, ay); return 0;
    }
    case O_EPL_MULTIPOLE_M1M3M4: {
      // reading: EPL_E1E2 (theta_E, gamma, e1, e2, cx, cy) plus the m = 1, 3, 4 multipoles about
      // the same centre with r_E = theta_E and phi_m = phi + dphi_m, phi = atan2(e2, e1)/2 the
      // EPL position angle; p = theta_E, gamma, e1, e2, cx, cy, a_1, dphi_1, a_3, dphi_3, a_4, dphi_4.
      T q, phi; e1e2_to_qphi(p[2], p[3], q, phi);
      alpha_epl(x, y, p[0], p[1], q, phi, p[4], p[5], ax, ay);
      const int ms[3] = {1, 3, 4};
      for (int i = 0; i < 3; ++i) {
        T mx, my;
        alpha_multipole(x, y, ms[i], p[6 + 2 * i], phi + p[7 + 2 * i], p[4], p[5], p[0], mx, my);
        ax += mx; ay += my;
      }
      return 0;
    }
    case O_CSE: {
      if constexpr (std::is_same<T, double>::value) {
        if (!(p[0] == p[0]) || !(p[1] > 0.0)) return -1;
        double q, phi; e1e2_to_qphi<double>(p[2], p[3], q, phi);
        alpha_cse(x, y, p[0], p[1], q, phi, p[4], p[5], ax, ay); return 0;
      } else {
        return -1;
      }
    }
    case O_MULTIPOLE_ELL: {
      if constexpr (std::is_same<T, double>::value) {
        const int m = (int)std::lround(p[0]);
        if (m < 1 || m > 32 || std::fabs(p[0] - m) > 1e-6 || !(p[3] >= 0.2 && p[3] <= 1.0) || !(p[7] > 0.0))
          return -1;
        alpha_multipole_ell(x, y, m, p[1], p[2], p[3], p[4], p[5], p[6], p[7], ax, ay);
        return 0;
      } else {
        return -1;
      }
    }
    case O_NFW_ELLIPSE_CSE:
    case O_HERNQUIST_ELLIPSE_CSE: {
      if constexpr (std::is_same<T, double>::value) {
        double q, phi; e1e2_to_qphi<double>(p[2], p[3], q, phi);
        if (type == O_NFW_ELLIPSE_CSE) {
          if (!(p[0] > 0.0)) return -1;
          alpha_nfw_ellipse(x, y, p[0], p[1], q, phi, p[4], p[5], ax, ay);
        } else {
          if (!(p[1] > 0.0)) return -1;
          alpha_hernquist_ellipse(x, y, p[0], p[1], q, phi, p[4], p[5], ax, ay);
        }
        return 0;
      } else {
        return -1;
      }
    }
    default: return -1;
  }
}

// ---------------------------------------------------------------------------
// Source light: elliptical Sersic (light table rows SERSIC, SERSIC_ELLIPSE,
// SERSIC_ELLIPSE_Q_PHI).
//   I = amp exp(-b_n [ (R/R_s)^(1/n) - 1 ]),  R = sqrt(q x'^2 + y'^2/q).
// reading: b_n = 1.9992 n - 0.3271 (Capaccioli 1989); amp is the brightness at R = R_s.
// ---------------------------------------------------------------------------
template <class T>
T sersic_I(const T& x, const T& y, const T& amp, const T& Rs, const T& n, const T& q, const T& phi,
           const T& cx, const T& cy) {
  T c = cos(phi), s = sin(phi);
  T dx = x - cx, dy = y - cy;
  T xp = c * dx + s * dy, yp = -s * dx + c * dy;
  T R = sqrt(q * xp * xp + yp * yp / q);
  T bn = 1.9992 * n - 0.3271;
  if (val(R) <= 0.0) return amp * exp(bn);
  T powv = exp(log(R / Rs) / n);
  return amp * exp(-bn * (powv - 1.0));
}

template <class T>
int light_profile(int type, const T* p, const T& x, const T& y, T& I) {
  switch (type) {
    case O_SERSIC_ELLIPSE_Q_PHI:
      I = sersic_I(x, y, p[0], p[1], p[2], p[3], p[4], p[5], p[6]); return 0;
    case O_SERSIC_ELLIPSE: {
      T q, phi; e1e2_to_qphi(p[3], p[4], q, phi);
      I = sersic_I(x, y, p[0], p[1], p[2], q, phi, p[5], p[6]); return 0;
    }
    case O_SERSIC:
      I = sersic_I(x, y, p[0], p[1], p[2], T(1.0), T(0.0), p[3], p[4]); return 0;
    default: return -1;
  }
}

// Cartesian shapelets (light table row SHAPELETS; Refregier 2003):
//   phi_n(u) = H_n(u) exp(-u^2/2) / sqrt(2^n n! sqrt(pi))   (H_n physicists' Hermite),
//   B_(n1,n2)(x, y) = phi_n1((x-cx)/beta) phi_n2((y-cy)/beta) / beta,   orthonormal in the plane,
//   I = sum_k amp_k B_(n1(k), n2(k)).
// reading: p = n_max, beta, cx, cy; the (n_max+1)(n_max+2)/2 amplitudes are ordered by
// n = n1 + n2 = 0, 1, ..., n_max and, within n, by n1 = n, n-1, ..., 0.
// H_n by its three-term recurrence H_(n+1) = 2u H_n - 2n H_(n-1), the normalisation as a product.
template <class T>
int shapelets_I(const T* p, const double* coef, int n_coef, const T& x, const T& y, T& I) {
  const int nmax = (int)std::lround(val(p[0]));
  if (nmax < 0 || nmax > 30 || n_coef != (nmax + 1) * (nmax + 2) / 2 || !(val(p[1]) > 0.0) || !coef) return -1;
  T u = (x - p[2]) / p[1], v = (y - p[3]) / p[1];
  std::vector<T> hu(nmax + 1), hv(nmax + 1);
  std::vector<double> norm(nmax + 1);
  hu[0] = T(1.0); hv[0] = T(1.0);
  if (nmax >= 1) { hu[1] = 2.0 * u; hv[1] = 2.0 * v; }
  for (int n = 1; n < nmax; ++n) {
    hu[n + 1] = 2.0 * u * hu[n] - 2.0 * n * hu[n - 1];
    hv[n + 1] = 2.0 * v * hv[n] - 2.0 * n * hv[n - 1];
  }
  double f = std::sqrt(std::sqrt(kPi));  // 2^n n! sqrt(pi), n = 0
  norm[0] = 1.0 / f;
  double prod = std::sqrt(kPi);
  for (int n = 1; n <= nmax; ++n) {
    prod *= 2.0 * n;
    norm[n] = 1.0 / std::sqrt(prod);
  }
  T sum = T(0.0);
  int k = 0;
  for (int n = 0; n <= nmax; ++n)
    for (int n1 = n; n1 >= 0; --n1, ++k) {
      const int n2 = n - n1;
      sum += coef[k] * norm[n1] * norm[n2] * hu[n1] * hv[n2];
    }
  I = sum * exp(-0.5 * (u * u + v * v)) / p[1];
  return 0;
}

// Any light profile: the table rows above, or shapelets with their amplitudes.
template <class T>
int source_I(int type, const T* p, const double* coef, int n_coef, const T& x, const T& y, T& I) {
  if (type == O_SHAPELETS) return shapelets_I(p, coef, n_coef, x, y, I);
  return light_profile(type, p, x, y, I);
}

inline double round32(double v) { return (double)(float)v; }
// Round the value of a number to FP32, keeping its tangents (conditioning-floor mode).
inline double r32(double v) { return round32(v); }
template <int N> inline Dual<N> r32(const Dual<N>& a) { Dual<N> r = a; r.v = round32(a.v); return r; }

}  // namespace

// ---------------------------------------------------------------------------
// C interface (ctypes).
// ---------------------------------------------------------------------------

extern "C" int oracle_nthreads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

extern "C" void oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

extern "C" int oracle_alpha(int type, const double* p, int n, const double* x, const double* y,
                 double* ax, double* ay) {
  for (int i = 0; i < n; ++i)
    if (alpha_profile<double>(type, p, x[i], y[i], ax[i], ay[i]) != 0) return -1;
  return 0;
}

extern "C" int oracle_light(int type, const double* p, const double* coef, int n_coef, int n, const double* x,
                            const double* y, double* I) {
  for (int i = 0; i < n; ++i)
    if (source_I<double>(type, p, coef, n_coef, x[i], y[i], I[i]) != 0) return -1;
  return 0;
}

// Grid (image simulation step 1).  reading: pixel (i, j) is centred at
//   x = x0 + (j - (nx-1)/2) dpix,  y = y0 + (i - (ny-1)/2) dpix   (+x right, row i = +y),
// and sub-pixel (a, b) of an s x s supersampling at offsets ((b + 1/2)/s - 1/2) dpix
// and ((a + 1/2)/s - 1/2) dpix.
static inline double grid_x(const oracle_system* S, int j, int b) {
  return S->x0 + (j - 0.5 * (S->nx - 1)) * S->dpix + ((b + 0.5) / S->s - 0.5) * S->dpix;
}
static inline double grid_y(const oracle_system* S, int i, int a) {
  return S->y0 + (i - 0.5 * (S->ny - 1)) * S->dpix + ((a + 0.5) / S->s - 0.5) * S->dpix;
}

// Total deflection at one point: the sum over the deflector list and over every
// subhalo (lens equation, image simulation step 1).  fp32 = 1 rounds each term to
// FP32 (the conditioning-floor mode) before the FP64 sum.
static int total_alpha(const oracle_system* S, double x, double y, int fp32, double& ax, double& ay) {
  ax = 0.0; ay = 0.0;
  for (int d = 0; d < S->n_defl; ++d) {
    double px, py;
    if (alpha_profile<double>(S->defl_type[d], S->defl_p + kDeflParams * d, x, y, px, py) != 0) return -1;
    if (fp32) { px = round32(px); py = round32(py); }
    ax += px; ay += py;
  }
  const int n = S->n_sub;
  for (int j = 0; j < n; ++j) {
    double px, py;
    alpha_tnfw<double>(x, y, S->sub[2 * n + j], S->sub[3 * n + j], S->sub[4 * n + j],
                       S->sub[j], S->sub[n + j], px, py);
    if (fp32) { px = round32(px); py = round32(py); }
    ax += px; ay += py;
  }
  return 0;
}

extern "C" int oracle_alpha_system(const oracle_system* S, int n, const double* x, const double* y,
                        double* ax, double* ay, int fp32) {
  int err = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : err)
  for (int i = 0; i < n; ++i) err |= total_alpha(S, x[i], y[i], fp32, ax[i], ay[i]) != 0;
  return err ? -1 : 0;
}

// Unconvolved image rows [row0, row1): steps 1-2 and the supersample bin-down.
// reading: a pixel holds the flux in it, dpix^2 times the mean of its s^2 samples.
extern "C" int oracle_image_rows(const oracle_system* S, int row0, int row1, double* out, int fp32) {
  if (row0 < 0 || row1 > S->ny || row0 > row1) return -1;
  const int nx = S->nx, s = S->s;
  int err = 0;
#pragma omp parallel for schedule(dynamic, 1) collapse(2) reduction(| : err)
  for (int i = row0; i < row1; ++i) {
    for (int j = 0; j < nx; ++j) {
      double sum = 0.0;
      for (int a = 0; a < s; ++a) {
        for (int b = 0; b < s; ++b) {
          double x = grid_x(S, j, b), y = grid_y(S, i, a);
          if (fp32) { x = round32(x); y = round32(y); }
          double ax, ay;
          err |= total_alpha(S, x, y, fp32, ax, ay) != 0;
          double bx = x - ax, by = y - ay;
          if (fp32) { bx = round32(bx); by = round32(by); }
          double I;
          err |= source_I<double>(S->src_type, S->src_p, S->src_coef, S->n_src_coef, bx, by, I) != 0;
          sum += I;
        }
      }
      out[(size_t)(i - row0) * nx + j] = sum * S->dpix * S->dpix / ((double)s * s);
    }
  }
  return err ? -1 : 0;
}

// PSF convolution (step 3), 'same' size, zero padding, odd k, c = (k-1)/2:
//   out[i][j] = sum_{a,b} K[a][b] img[i + c - a][j + c - b].
template <class T>
static void convolve_same(const T* img, int ny, int nx, const double* K, int k, T* out) {
  const int c = (k - 1) / 2;
  for (int i = 0; i < ny; ++i)
    for (int j = 0; j < nx; ++j) {
      T acc = T(0.0);
      for (int a = 0; a < k; ++a) {
        int ii = i + c - a;
        if (ii < 0 || ii >= ny) continue;
        for (int b = 0; b < k; ++b) {
          int jj = j + c - b;
          if (jj < 0 || jj >= nx) continue;
          acc += K[a * k + b] * img[(size_t)ii * nx + jj];
        }
      }
      out[(size_t)i * nx + j] = acc;
    }
}

extern "C" int oracle_convolve(const double* img, int ny, int nx, const double* K, int k, double* out) {
  if (k <= 0 || (k % 2) == 0) return -1;
  convolve_same<double>(img, ny, nx, K, k, out);
  return 0;
}

// Transpose of the zero-padded 'same' convolution: correlation with K,
//   out[i][j] = sum_{a,b} K[a][b] img[i - c + a][j - c + b].
extern "C" int oracle_correlate(const double* img, int ny, int nx, const double* K, int k, double* out) {
  if (k <= 0 || (k % 2) == 0) return -1;
  const int c = (k - 1) / 2;
  for (int i = 0; i < ny; ++i)
    for (int j = 0; j < nx; ++j) {
      double acc = 0.0;
      for (int a = 0; a < k; ++a) {
        int ii = i - c + a;
        if (ii < 0 || ii >= ny) continue;
        for (int b = 0; b < k; ++b) {
          int jj = j - c + b;
          if (jj < 0 || jj >= nx) continue;
          acc += K[a * k + b] * img[(size_t)ii * nx + jj];
        }
      }
      out[(size_t)i * nx + j] = acc;
    }
  return 0;
}

// Full image: unconvolved rows, then the PSF (if any).
extern "C" int oracle_image(const oracle_system* S, double* out, double* unconvolved, int fp32) {
  std::vector<double> raw((size_t)S->nx * S->ny);
  if (oracle_image_rows(S, 0, S->ny, raw.data(), fp32) != 0) return -1;
  if (unconvolved) std::memcpy(unconvolved, raw.data(), raw.size() * sizeof(double));
  if (S->k > 0) return oracle_convolve(raw.data(), S->ny, S->nx, S->psf, S->k, out);
  std::memcpy(out, raw.data(), raw.size() * sizeof(double));
  return 0;
}

// ---------------------------------------------------------------------------
// Chi^2 log-likelihood and its exact gradient (15 free parameters).
// Parameter order: main deflector EPL (theta_E, gamma, e1, e2, cx, cy), shear (g1, g2),
// source SERSIC_ELLIPSE (amp, R_s, n, e1, e2, cx, cy).  The subhalo deflections are
// held fixed.  reading: the pixel variance is model-dependent,
//   sigma^2 = sigma_bkg^2 + max(m, 0) / t_exp,   logL = -1/2 sum (d - m)^2 / sigma^2,
// with no log-determinant term (paper: "a variety of log-likelihood functions").
// ---------------------------------------------------------------------------
constexpr int kNP = 15;
using D15 = Dual<kNP>;

// fp32 = 1: conditioning-floor mode; the grid, every deflection term, the traced position and
// the model image are rounded to FP32 (values only, tangents kept).
template <class T>
static double loglike_T(const oracle_system* S, const double* data, double sigma_bkg, double t_exp,
                        const std::vector<double>& asx, const std::vector<double>& asy,
                        const T* P, T* logL_out, int fp32) {
  const int nx = S->nx, ny = S->ny, s = S->s;
  std::vector<T> raw((size_t)nx * ny), model((size_t)nx * ny);
  const double w = S->dpix * S->dpix / ((double)s * s);
  T epl[6] = {P[0], P[1], P[2], P[3], P[4], P[5]};
  T src[7] = {P[8], P[9], P[10], P[11], P[12], P[13], P[14]};
  for (int i = 0; i < ny; ++i)
    for (int j = 0; j < nx; ++j) {
      T sum = T(0.0);
      for (int a = 0; a < s; ++a)
        for (int b = 0; b < s; ++b) {
          size_t sp = (((size_t)i * nx + j) * s + a) * s + b;
          double x = grid_x(S, j, b), y = grid_y(S, i, a);
          double ux = asx[sp], uy = asy[sp];
          if (fp32) { x = round32(x); y = round32(y); ux = round32(ux); uy = round32(uy); }
          T ax, ay, sx, sy;
          alpha_profile<T>(O_EPL_E1E2, epl, T(x), T(y), ax, ay);
          alpha_shear<T>(T(x), T(y), P[6], P[7], sx, sy);
          if (fp32) { ax = r32(ax); ay = r32(ay); sx = r32(sx); sy = r32(sy); }
          T bx = T(x) - ax - sx - ux;
          T by = T(y) - ay - sy - uy;
          if (fp32) { bx = r32(bx); by = r32(by); }
          T I;
          light_profile<T>(O_SERSIC_ELLIPSE, src, bx, by, I);
          sum += I;
        }
      raw[(size_t)i * nx + j] = sum * w;
    }
  if (S->k > 0) convolve_same<T>(raw.data(), ny, nx, S->psf, S->k, model.data());
  else model = raw;
  T acc = T(0.0);
  const double vb = sigma_bkg * sigma_bkg;
  for (size_t p = 0; p < model.size(); ++p) {
    T m = fp32 ? r32(model[p]) : model[p];
    T var = (val(m) > 0.0) ? vb + m / t_exp : T(vb);
    T r = data[p] - m;
    acc += r * r / var;
  }
  *logL_out = -0.5 * acc;
  return val(*logL_out);
}

// Fixed subhalo deflection at every sub-pixel sample, in sample order (i, j, a, b).
static void subhalo_field(const oracle_system* S, std::vector<double>& asx, std::vector<double>& asy) {
  const int nx = S->nx, ny = S->ny, s = S->s, n = S->n_sub;
  size_t total = (size_t)nx * ny * s * s;
  asx.assign(total, 0.0); asy.assign(total, 0.0);
#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < ny; ++i)
    for (int j = 0; j < nx; ++j)
      for (int a = 0; a < s; ++a)
        for (int b = 0; b < s; ++b) {
          size_t sp = (((size_t)i * nx + j) * s + a) * s + b;
          double x = grid_x(S, j, b), y = grid_y(S, i, a), ax = 0.0, ay = 0.0;
          for (int k = 0; k < n; ++k) {
            double px, py;
            alpha_tnfw<double>(x, y, S->sub[2 * n + k], S->sub[3 * n + k], S->sub[4 * n + k],
                               S->sub[k], S->sub[n + k], px, py);
            ax += px; ay += py;
          }
          asx[sp] = ax; asy[sp] = ay;
        }
}

// params: [n_points][15]; logL: [n_points]; grad: [n_points][15] or NULL.
extern "C" int oracle_loglike(const oracle_system* S, const double* data, double sigma_bkg, double t_exp,
                   const double* params, int n_points, double* logL, double* grad, int fp32) {
  std::vector<double> asx, asy;
  subhalo_field(S, asx, asy);
#pragma omp parallel for schedule(dynamic, 1)
  for (int p = 0; p < n_points; ++p) {
    const double* P = params + (size_t)p * kNP;
    if (grad) {
      D15 Pd[kNP];
      for (int k = 0; k < kNP; ++k) { Pd[k] = D15(P[k]); Pd[k].d[k] = 1.0; }
      D15 L;
      loglike_T<D15>(S, data, sigma_bkg, t_exp, asx, asy, Pd, &L, fp32);
      logL[p] = L.v;
      for (int k = 0; k < kNP; ++k) grad[(size_t)p * kNP + k] = L.d[k];
    } else {
      double L;
      loglike_T<double>(S, data, sigma_bkg, t_exp, asx, asy, P, &L, fp32);
      logL[p] = L;
    }
  }
  return 0;
}

// Model image (PSF-convolved) at one 15-parameter point, for generating observations.
extern "C" int oracle_model_image(const oracle_system* S, const double* params, double* out) {
  std::vector<double> asx, asy;
  subhalo_field(S, asx, asy);
  const int nx = S->nx, ny = S->ny;
  const int s = S->s;
  const double w = S->dpix * S->dpix / ((double)s * s);
  std::vector<double> raw((size_t)nx * ny);
  const double* P = params;
  for (int i = 0; i < ny; ++i)
    for (int j = 0; j < nx; ++j) {
      double sum = 0.0;
      for (int a = 0; a < s; ++a)
        for (int b = 0; b < s; ++b) {
          size_t sp = (((size_t)i * nx + j) * s + a) * s + b;
          double x = grid_x(S, j, b), y = grid_y(S, i, a), ax, ay, sx, sy, I;
          alpha_profile<double>(O_EPL_E1E2, P, x, y, ax, ay);
          alpha_shear<double>(x, y, P[6], P[7], sx, sy);
          light_profile<double>(O_SERSIC_ELLIPSE, P + 8, x - ax - sx - asx[sp], y - ay - sy - asy[sp], I);
          sum += I;
        }
      raw[(size_t)i * nx + j] = sum * w;
    }
  if (S->k > 0) return oracle_convolve(raw.data(), ny, nx, S->psf, S->k, out);
  std::memcpy(out, raw.data(), raw.size() * sizeof(double));
  return 0;
}


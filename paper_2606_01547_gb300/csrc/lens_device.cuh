// Device-side FP32 lensing arithmetic for sm_103a: deflection profiles, the truncated-NFW
// subhalo pair term, and the elliptical Sersic source.  Every accumulation is FP32; no FP64
// is used on the device.
//
// Profiles follow their published definitions (the paper names them in its deflection and
// light tables but prints no formula):
//   SIE   Kormann, Schneider & Bartelmann (1994): kappa = theta_E / (2 sqrt(q x'^2 + y'^2/q)).
//   EPL   Tessore & Metcalf (2015): hypergeometric series in e^{2 i phi}, b = theta_E sqrt(q).
//   NFW   Bartelmann (1996), Wright & Brainerd (2000); alpha_Rs = deflection at r = Rs.
//   TNFW  Baltz, Marshall & Oguri (2009), n = 1 truncation, tau = r_t / Rs.
//   Sersic I = amp exp(-b_n [(R/R_s)^(1/n) - 1]), R = sqrt(q x'^2 + y'^2/q), b_n = 1.9992 n - 0.3271.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lens_sim.h"
#include "cse_fits.h"

namespace ls {

constexpr float kPi = 3.14159265358979323846f;
constexpr float kHalfPi = 1.57079632679489661923f;
constexpr float kLn2 = 0.69314718055994530942f;
constexpr float kOneMinusLn2 = 0.30685281944005469058f;

struct DevProfile {
  int type;
  float p[LENS_PROFILE_PARAMS];
};

// One lens system as the kernels see it.  `sub` is the precomputed table of its n_sub subhalos
// (kTableStride float4 per subhalo, see tnfw_write_table); `out` receives the binned,
// unconvolved image.
// Harmonics kept for the elliptical multipole (enough for 1e-8 of the largest coefficient at
// m <= 32, q >= 0.2, where the series needs at most 314).
constexpr int kEllMaxK = 320;
constexpr int kEllTableFloats = 2 * (kEllMaxK + 1);

struct DevSystem {
  int nx, ny, s, n_defl;
  float dpix, x0, y0;
  int src_type;
  float src[8];
  float src_coef[LENS_MAX_SHAPELET_COEFFS];  // SHAPELETS amplitudes
  int ell_K;                                 // LENS_MULTIPOLE_ELL: harmonics 0..ell_K of 2 kappa r
  const float* ell_c;                        // in device memory, (Re, Im) pairs scaled by a_m r_E
                                             // (nullptr without the profile)
  DevProfile defl[LENS_MAX_DEFLECTORS];
  int n_sub;
  float far_kappa;  // > 0: far-field interpolation of the subhalo sum from kappa box half-widths
  const float4* sub;
  float* out;
};

// ---------------------------------------------------------------------------- helpers
__device__ __forceinline__ void e1e2_to_qphi(float e1, float e2, float& q, float& phi) {
  phi = 0.5f * atan2f(e2, e1);
  float c = sqrtf(e1 * e1 + e2 * e2);
  q = (1.f - c) / (1.f + c);
}

__device__ __forceinline__ void to_frame(float dx, float dy, float cp, float sp, float& xp, float& yp) {
  xp = cp * dx + sp * dy;
  yp = -sp * dx + cp * dy;
}

// ---------------------------------------------------------------------------- main deflectors
__device__ __forceinline__ void alpha_sis(float x, float y, float thetaE, float cx, float cy,
                                          float& ax, float& ay) {
  float dx = x - cx, dy = y - cy;
  float r2 = dx * dx + dy * dy;
  if (r2 < 1e-24f) { ax = 0.f; ay = 0.f; return; }
  float ir = rsqrtf(r2);
  ax = thetaE * dx * ir;
  ay = thetaE * dy * ir;
}

__device__ __forceinline__ void alpha_point_mass(float x, float y, float thetaE, float cx, float cy,
                                                 float& ax, float& ay) {
  float dx = x - cx, dy = y - cy;
  float r2 = dx * dx + dy * dy;
  if (r2 < 1e-24f) { ax = 0.f; ay = 0.f; return; }
  float k = thetaE * thetaE / r2;
  ax = k * dx;
  ay = k * dy;
}

static __device__ __noinline__ void alpha_sie(float x, float y, float thetaE, float q, float phi, float cx,
                                       float cy, float& ax, float& ay) {
  float sp, cp;
  sincosf(phi, &sp, &cp);
  float dx = x - cx, dy = y - cy, xp, yp;
  to_frame(dx, dy, cp, sp, xp, yp);
  float r2 = dx * dx + dy * dy;
  if (r2 < 1e-24f) { ax = 0.f; ay = 0.f; return; }
  float apx, apy;
  if (fabsf(1.f - q) < 1e-6f) {
    float ir = rsqrtf(r2);
    apx = thetaE * xp * ir;
    apy = thetaE * yp * ir;
  } else {
    float b = thetaE * sqrtf(q);
    float psi = sqrtf(q * q * xp * xp + yp * yp);
    float e = sqrtf((1.f - q) * (1.f + q));
    float be = b / e;
    apx = be * atanf(e * xp / psi);
    apy = be * atanhf(e * yp / psi);
  }
  ax = cp * apx - sp * apy;
  ay = sp * apx + cp * apy;
}

// Number of EPL series terms for FP32: |Omega_n| <= f^n, stop once f^n < 2^-26.
__device__ __forceinline__ int epl_terms(float f) {
  if (f < 1e-20f) return 0;
  int n = (int)ceilf(-18.0218f / logf(f)) + 1;
  return n < 1 ? 1 : (n > 200 ? 200 : n);
}

// EPL (Tessore & Metcalf 2015): the quantities of one lens that do not depend on the point
// (its frame), and the deflection at a point from them, with the series coefficients
// c_n = (2n - 2 + t)/(2n + 2 - t) taken from `coef(n)`: computed in place by alpha_epl, read
// from a per-point table by the likelihood kernels (which also keep one frame per point).
struct EplFrame {
  float cp, sp;  // cos, sin of the position angle
  float q, t;    // axis ratio, gamma - 1
  float b, f;    // theta_E sqrt(q), (1 - q)/(1 + q)
  float b2q;     // 2 b / (1 + q)
  int nt;        // series terms
};

__device__ __forceinline__ EplFrame epl_frame(float thetaE, float gamma, float q, float phi) {
  EplFrame e;
  sincosf(phi, &e.sp, &e.cp);
  e.q = q;
  e.t = gamma - 1.f;
  e.b = thetaE * sqrtf(q);
  e.f = (1.f - q) / (1.f + q);
  e.b2q = 2.f * e.b / (1.f + q);
  e.nt = epl_terms(e.f);
  return e;
}

template <class Coef>
__device__ __forceinline__ void alpha_epl_at(float x, float y, const EplFrame& e, float cx, float cy, Coef coef,
                                             float& ax, float& ay) {
  float dx = x - cx, dy = y - cy, xp, yp;
  to_frame(dx, dy, e.cp, e.sp, xp, yp);
  float R = sqrtf(e.q * e.q * xp * xp + yp * yp);
  if (R < 1e-12f) { ax = 0.f; ay = 0.f; return; }
  float iR = 1.f / R;
  float er = e.q * xp * iR, ei = yp * iR;
  float zr = -e.f * (er * er - ei * ei), zi = -e.f * (2.f * er * ei);
  float omr = er, omi = ei, sr = er, si = ei;
  for (int n = 1; n <= e.nt; ++n) {
    const float c = coef(n);
    float nr = c * (omr * zr - omi * zi);
    float ni = c * (omr * zi + omi * zr);
    omr = nr; omi = ni;
    sr += omr; si += omi;
  }
  float pref = e.b2q * exp2f((e.t - 1.f) * log2f(e.b * iR));
  float apx = pref * sr, apy = pref * si;
  ax = e.cp * apx - e.sp * apy;
  ay = e.sp * apx + e.cp * apy;
}

__device__ __forceinline__ float epl_coef(int n, float t) { return (2.f * n - 2.f + t) / (2.f * n + 2.f - t); }

static __device__ __noinline__ void alpha_epl(float x, float y, float thetaE, float gamma, float q, float phi,
                                       float cx, float cy, float& ax, float& ay) {
  const EplFrame e = epl_frame(thetaE, gamma, q, phi);
  const float t = e.t;
  alpha_epl_at(x, y, e, cx, cy, [t](int n) { return epl_coef(n, t); }, ax, ay);
}

// ---------------------------------------------------------------------------- NFW / TNFW
// Both are written as alpha = K * g(x^2) * (dx, dy) with x = r/Rs and g = M(x)/x^2 up to a
// constant; the functions below return that g for FP32 without catastrophic cancellation.

// F(x) near x = 1 as sum_k (-v)^k/(2k+1), v = x^2 - 1 (|v| < 0.1: 9 terms reach 1e-10).
__device__ __forceinline__ float nfw_F_series(float v) {
  float s = 0.f, t = 1.f;
#pragma unroll
  for (int k = 0; k < 9; ++k) { s += t / (2.f * k + 1.f); t *= -v; }
  return s;
}

__device__ __forceinline__ float nfw_F(float x2) {
  float v = x2 - 1.f;
  if (fabsf(v) < 0.1f) return nfw_F_series(v);
  if (v > 0.f) { float u = sqrtf(v); return atanf(u) / u; }
  float x = sqrtf(x2);
  float u = sqrtf((1.f - x) * (1.f + x));
  return logf((1.f + u) / x) / u;
}

// NFW: h(x)/x^2 with h = ln(x/2) + F(x).  For x < 1, with u = sqrt(1-x^2), w = 1-u = x^2/(1+u):
// h = [log1p(-w/2) + w ln(2/x)] / u, whose two terms are both O(x^2).
static __device__ __noinline__ float nfw_h_over_x2(float x2) {
  if (x2 < 0.81f) {
    float x = sqrtf(x2);
    float u = sqrtf((1.f - x) * (1.f + x));
    float wx = 1.f / (1.f + u);       // w / x^2
    float w = x2 * wx;
    float z = -0.5f * w;
    float l1 = (log1pf(z) / z) * (-0.5f * wx);  // log1p(-w/2) / x^2
    return (l1 + (kLn2 - logf(x)) * wx) / u;
  }
  float x = sqrtf(x2);
  return (logf(0.5f * x) + nfw_F(x2)) / x2;
}

// Taylor coefficients of asin(y)/y = sum_k c_k y^(2k), c_k = (2k)! / (4^k (k!)^2 (2k+1));
// asinh(z)/z is the same series with alternating signs.
__device__ __forceinline__ float asin_over_y(float y2) {
  float p = 0.017352764f;                 // 231/13312
  p = fmaf(p, y2, 0.022372159f);          // 63/2816
  p = fmaf(p, y2, 0.030381944f);          // 35/1152
  p = fmaf(p, y2, 0.044642857f);          // 5/112
  p = fmaf(p, y2, 0.075f);                // 3/40
  p = fmaf(p, y2, 0.16666667f);           // 1/6
  return fmaf(p, y2, 1.f);
}

__device__ __forceinline__ float asinh_over_z(float z2) {
  float p = 0.017352764f;
  p = fmaf(p, -z2, 0.022372159f);
  p = fmaf(p, -z2, 0.030381944f);
  p = fmaf(p, -z2, 0.044642857f);
  p = fmaf(p, -z2, 0.075f);
  p = fmaf(p, -z2, 0.16666667f);
  return fmaf(p, -z2, 1.f);
}

// Truncated NFW bracket G(x) of M(x) = tau^2/(tau^2+1)^2 G(x):
//   G = (tau^2 + 1 + 2(x^2-1)) F(x) + tau pi + (tau^2-1) ln tau + S (-pi + L (tau^2-1)/tau),
//   S = sqrt(tau^2 + x^2),  L = ln(x / (S + tau)) = -asinh(tau/x).
// Returned: G/x^2.  Constants: t2 = tau^2, t2m1 = tau^2 - 1, C = tau pi + (tau^2-1) ln tau.
//
// Three evaluation regimes, each free of catastrophic cancellation in FP32:
//  x < 0.9  : G = (tau^2-1) D + 2 x^2 F + pi (tau - S), D = F + ln tau + (S/tau) L, with D and
//             tau - S rewritten as sums of O(x^2) terms (log1p forms);
//  x < 4    : the defining formula (cancellation is mild there);
//  x >= 4   : in y = 1/x, z = tau y, r1 = (1-y^2)^(-1/2), Sx = sqrt(1+z^2), P = asin(y)/y:
//             G = r1 [(tau^2-1)(pi/2 y - y^2 P) - 2P] + C + pi y (tau^2 y^2 - (tau^2-1)) r1^2/(r1+Sx)
//                 - (tau^2-1) Sx asinh(z)/z,
//             which removes the +-pi x cancellation and the ln of a ratio near 1.
static __device__ __noinline__ float tnfw_g_near(float x2, float tau, float t2, float t2m1, float C) {
  float S = sqrtf(t2 + x2);
  if (x2 < 0.81f) {
    float x = sqrtf(x2);
    float u = sqrtf((1.f - x) * (1.f + x));
    float wx = 1.f / (1.f + u);
    float w = x2 * wx;
    float lnx = logf(x);
    float F = logf((1.f + u) / x) / u;
    float L = -asinhf(tau / x);
    float z = -0.5f * w;
    float l1 = (log1pf(z) / z) * (-0.5f * wx);
    float l2 = log1pf(x2 / (2.f * tau * (S + tau))) / x2;
    float Dx2 = (l1 + (kLn2 - lnx) * wx) / u - l2 + L / (tau * (S + tau));
    return t2m1 * Dx2 + 2.f * F - kPi / (tau + S);
  }
  float F = nfw_F(x2);
  float x = sqrtf(x2);
  float L = -asinhf(tau / x);
  float G = (t2m1 + 2.f * x2) * F + C + S * (-kPi + L * t2m1 / tau);
  return G / x2;
}

__device__ __forceinline__ float tnfw_g_far(float x2, float tau, float t2, float t2m1, float C) {
  float y = rsqrtf(x2);
  float y2 = y * y;
  float r1 = rsqrtf(1.f - y2);
  float z = tau * y;
  float z2 = z * z;
  float sq = 1.f + z2;
  float Sx = sq * rsqrtf(sq);
  float P = asin_over_y(y2);
  float ash = (z2 < 0.0625f) ? asinh_over_z(z2) : __fdividef(logf(z + Sx), z);
  float head = r1 * fmaf(t2m1, fmaf(kHalfPi, y, -y2 * P), -2.f * P);
  float mid = __fdividef(kPi * y * fmaf(t2, y2, -t2m1) * r1 * r1, r1 + Sx);
  float G = head + C + mid - t2m1 * Sx * ash;
  return G * y2;
}


// ---------------------------------------------------------------------------- subhalo table
// Far field (x >= 7 max(tau, 1)): G(x) is analytic in y = 1/x for |y| < min(1, 1/tau), and
//   G = sum_k c_k y^k,  c_0 = C - (tau^2 + 1),  c_1 = 0,
//   c_(2n+1) = pi [ (tau^2-1) a_n / 2 + a_(n+1) - s_(n+1) tau^(2n+2) ],
//   c_(2n)   = -(tau^2-1) b_(n-1) - 2 b_n - (tau^2-1) tau^(2n) sum_(i+j=n) s_i h_j,
// from the Taylor series of (1-y^2)^(-1/2) = sum a_j y^2j, asin(y)/sqrt(1-y^2) = sum b_j y^(2j+1),
// sqrt(1+u) = sum s_j u^j and asinh(z) = sum h_j z^(2j+1) substituted into the defining formula
// (the 1/y terms cancel exactly).  Truncated after c_6 and used from x >= kFarRadius max(tau, 1)
// = 7 max(tau, 1) on, the relative error is below 1e-6 for all tau (FP32 closed forms reach
// 3e-6), and Horner in FP32 is well conditioned (sum |c_k y^k| / |G| < 1.1).
constexpr int kFarTerms = 6;
constexpr float kFarRadius = 7.f;  // the series' range: r >= kFarRadius max(tau, 1) Rs
static_assert(kFarTerms >= 3 && kFarTerms <= 6, "the record holds d_0, d_2 .. d_6 in t2..t4");
// Farther out the series converges faster, so fewer terms reach the same accuracy (largest
// relative truncation error over tau in [0.1, 30], in FP64 against the closed form):
//   c_0 .. c_6 from 7 max(tau, 1) Rs: 9.5e-7;  c_0 .. c_4 from 20: 2.3e-7;  c_0 .. c_3 from 40: 3.6e-7.
// A subhalo takes the shortest series whose range holds every sample of a unit (its distance
// to the unit's bounding box decides).
constexpr float kFarRadius4 = 20.f;  // 4-term series (c_0, c_2, c_3, c_4) from here
constexpr float kFarRadius3 = 40.f;  // 3-term series (c_0, c_2, c_3) from here
constexpr int kSubStride = 8;   // float4 per subhalo record (staged through shared memory)
constexpr int kMidTerms = 12;   // coefficients of the annulus polynomial
constexpr int kMidStride = 3;   // float4 per subhalo in the annulus block
constexpr int kFarStride = 3;   // float4 per subhalo in the compact far-field block
constexpr int kTableStride = kSubStride + kMidStride + kFarStride;  // float4 per subhalo in a whole table
// Largest tau whose annulus 4 <= x < 7 max(tau, 1) the 12-term polynomial covers to 1e-7
// (relative, in FP64 arithmetic); beyond it the annulus takes the closed form.
constexpr float kMidTauMax = 8.5f;

// A subhalo table of n subhalos is n records of kSubStride float4, then n annulus blocks of
// kMidStride float4, then n compact far-field blocks of kFarStride float4,
//   f0 = (-cx, -cy, r_far^2, r_4^2),  f1 = (r_3^2, d_0, d_2, d_3),  f2 = (d_4, d_5, d_6, 0),
// the same numbers as the record's, once each: all that the bounding-box test and the far-field
// series read, in 48 B instead of 128 B (the image kernels stage the table once per unit and
// slice).  The record (128 B) is laid out for packed FP32x2 arithmetic (two samples
// per instruction): centres negated and every series coefficient stored as a duplicated pair,
//   t0 = (-cx, -cx, -cy, -cy),           t1 = (r_far^2 = 49 max(tau,1)^2 Rs^2, 1/Rs^2, tau, A),
//   t2 = (d_0, d_0, d_2, d_2),  t3 = (d_3, d_3, d_4, d_4),  t4 = (d_5, d_5, d_6, d_6),
//   t5 = (r_4^2, r_3^2, 0, 0): the ranges of the 4- and 3-term series (kFarRadius4 and
//   kFarRadius3 times max(tau, 1) Rs, squared),  t6 = (a_t, b_t, r_in^2, C),  t7 = 0,
// with A = alpha_Rs tau^2 / ((1 - ln 2) Rs (tau^2+1)^2), so that alpha = A g(x^2) (dx, dy), and
// d_k = A c_k Rs^(k+2): the series then runs in u = 1/r with no per-pair scaling by 1/Rs^2.
// C = tau pi + (tau^2-1) ln tau.  The annulus block holds the 12 coefficients e_0..e_11 of
//   A g = u^2 sum_j e_j t^j,  t = a_t u + b_t,
// the polynomial in t in [-1, 1] that interpolates A Rs^2 G at the 12 Chebyshev nodes of
// y = Rs u in [1/(7 max(tau, 1)), 1/4], i.e. on the annulus r_in = 4 Rs <= r < r_far.  When the
// annulus is too wide for 12 terms (tau > kMidTauMax), r_in^2 = r_far^2 and the block is zero.
__device__ __forceinline__ void tnfw_constants(float cx, float cy, float Rs, float alphaRs, float rt, float4* t) {
  const float tau = rt / Rs;
  const float t2 = tau * tau, t2m1 = t2 - 1.f, t2p1 = t2 + 1.f;
  const float A = alphaRs * t2 / (kOneMinusLn2 * Rs * t2p1 * t2p1);
  const float C = tau * kPi + t2m1 * logf(tau);
  float a[7], b[7], sq[7], h[7];
  a[0] = 1.f; b[0] = 1.f; sq[0] = 1.f;
  for (int j = 0; j < 6; ++j) {
    a[j + 1] = a[j] * (2.f * j + 1.f) / (2.f * j + 2.f);
    b[j + 1] = b[j] * (2.f * j + 2.f) / (2.f * j + 3.f);
    sq[j + 1] = sq[j] * (0.5f - j) / (j + 1.f);
  }
  for (int j = 0; j < 7; ++j) h[j] = ((j & 1) ? -a[j] : a[j]) / (2.f * j + 1.f);
  float c[kFarTerms + 1];
  c[0] = C - t2p1;
  c[1] = 0.f;
  float t2pow = t2;  // tau^(2n) for the even terms, advanced below
  for (int n = 1; 2 * n <= kFarTerms; ++n) {
    float P = 0.f;
    for (int i = 0; i <= n; ++i) P += sq[i] * h[n - i];
    c[2 * n] = -t2m1 * b[n - 1] - 2.f * b[n] - t2m1 * t2pow * P;
    if (2 * n + 1 <= kFarTerms) c[2 * n + 1] = kPi * (0.5f * t2m1 * a[n] + a[n + 1] - sq[n + 1] * t2pow * t2);
    t2pow *= t2;
  }
  float d[kFarTerms + 1];
  float rp = Rs * Rs;  // Rs^(k+2)
  for (int k = 0; k <= kFarTerms; ++k) {
    d[k] = A * c[k] * rp;
    rp *= Rs;
  }
  const float tm = fmaxf(tau, 1.f);
  const float r_far2 = kFarRadius * kFarRadius * tm * tm * Rs * Rs;
  const bool annulus = tau <= kMidTauMax;
  // t = (2y - (ylo + yhi)) / (yhi - ylo) with y = Rs u, ylo = 1/(7 max(tau, 1)), yhi = 1/4
  const float ylo = 1.f / (kFarRadius * tm), yhi = 0.25f;
  const float at = annulus ? 2.f * Rs / (yhi - ylo) : 0.f;
  const float bt = annulus ? -(ylo + yhi) / (yhi - ylo) : 0.f;
  t[0] = make_float4(-cx, -cx, -cy, -cy);
  t[1] = make_float4(r_far2, 1.f / (Rs * Rs), tau, A);
  float seq[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // d_0, d_2, ..., d_kFarTerms
  seq[0] = d[0];
  for (int k = 2; k <= kFarTerms; ++k) seq[k - 1] = d[k];
  for (int j = 0; j < 3; ++j) t[2 + j] = make_float4(seq[2 * j], seq[2 * j], seq[2 * j + 1], seq[2 * j + 1]);
  const float tmR = tm * Rs;
  t[5] = make_float4(kFarRadius4 * kFarRadius4 * tmR * tmR, kFarRadius3 * kFarRadius3 * tmR * tmR, 0.f, 0.f);
  t[6] = make_float4(at, bt, annulus ? 16.f * Rs * Rs : r_far2, C);
  t[7] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Annulus block of a subhalo from its record t (Rs = its scale radius): G at the 12 Chebyshev
// nodes of y in [1/(7 max(tau, 1)), 1/4] by the x >= 4 closed form, Chebyshev coefficients by the
// discrete cosine sum, then the monomial coefficients in t (T_j expanded by its recurrence,
// whose integer coefficients are exact in FP32; the monomial form's FP32 condition number on
// [-1, 1] is below 2 for tau <= kMidTauMax), scaled by A Rs^2.
__device__ __forceinline__ void tnfw_mid_constants(float Rs, const float4* t, float4* m) {
  float e[kMidTerms];
#pragma unroll
  for (int j = 0; j < kMidTerms; ++j) e[j] = 0.f;
  if (t[6].z < t[1].x) {
    const float tau = t[1].z, A = t[1].w, C = t[6].w;
    const float t2 = tau * tau, t2m1 = t2 - 1.f;
    const float ylo = 1.f / (kFarRadius * fmaxf(tau, 1.f)), yhi = 0.25f;
    float ch[kMidTerms];
#pragma unroll
    for (int j = 0; j < kMidTerms; ++j) ch[j] = 0.f;
#pragma unroll
    for (int k = 0; k < kMidTerms; ++k) {
      const float tk = cospif((k + 0.5f) / kMidTerms);
      const float y = fmaf(0.5f * (yhi - ylo), tk, 0.5f * (yhi + ylo));
      const float x2 = 1.f / (y * y);
      const float G = tnfw_g_far(x2, tau, t2, t2m1, C) * x2;
      float Tm = 1.f, Tj = tk;  // T_0, T_1 at the node
      ch[0] += G;
      ch[1] += G * tk;
#pragma unroll
      for (int j = 2; j < kMidTerms; ++j) {
        const float Tn = fmaf(2.f * tk, Tj, -Tm);
        ch[j] += G * Tn;
        Tm = Tj;
        Tj = Tn;
      }
    }
#pragma unroll
    for (int j = 0; j < kMidTerms; ++j) ch[j] *= (j == 0 ? 1.f : 2.f) / kMidTerms;
    // monomial coefficients: e += ch_j * T_j, with T_j's coefficients from T_(j+1) = 2t T_j - T_(j-1)
    float Tp[kMidTerms], Tc[kMidTerms];
#pragma unroll
    for (int i = 0; i < kMidTerms; ++i) { Tp[i] = 0.f; Tc[i] = 0.f; }
    Tp[0] = 1.f;  // T_0
    Tc[1] = 1.f;  // T_1
    e[0] = ch[0];
    e[1] = ch[1];
#pragma unroll
    for (int j = 2; j < kMidTerms; ++j) {
#pragma unroll
      for (int i = kMidTerms - 1; i >= 0; --i) {
        const float Tn = (i > 0 ? 2.f * Tc[i - 1] : 0.f) - Tp[i];
        Tp[i] = Tc[i];
        Tc[i] = Tn;
      }
#pragma unroll
      for (int i = 0; i < kMidTerms; ++i) e[i] = fmaf(ch[j], Tc[i], e[i]);
    }
    const float s = A * Rs * Rs;
#pragma unroll
    for (int j = 0; j < kMidTerms; ++j) e[j] *= s;
  }
  m[0] = make_float4(e[0], e[1], e[2], e[3]);
  m[1] = make_float4(e[4], e[5], e[6], e[7]);
  m[2] = make_float4(e[8], e[9], e[10], e[11]);
}

// Reciprocal square root on the MUFU with flush-to-zero: every argument it gets is at least
// 16 Rs^2 > 0 and never denormal, so the IEEE-mode rsqrtf fix-up is not needed.
__device__ __forceinline__ float rsqrt_ftz(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Series coefficient d_k of a record (k = 0 or 2..kFarTerms): the sequence d_0, d_2, d_3, ...
// fills t2, t3, ... two per float4, each as a duplicated pair (x, y) or (z, w).
__device__ __forceinline__ int tnfw_coef_slot(int k) { return k == 0 ? 0 : k - 1; }
__device__ __forceinline__ float tnfw_coef(const float4* t, int k) {
  const int e = tnfw_coef_slot(k);
  return (e & 1) ? t[2 + e / 2].z : t[2 + e / 2].x;
}
__device__ __forceinline__ float2 tnfw_coef2(const float4* t, int k) {
  const int e = tnfw_coef_slot(k);
  const float4 v = t[2 + e / 2];
  return (e & 1) ? make_float2(v.z, v.w) : make_float2(v.x, v.y);
}

// Far-field series: A g = u^2 (d_0 + u^2 (d_2 + d_3 u + ... + d_6 u^4)), u = 1/r, u2 = u^2,
// the same as A y^2 sum_k c_k y^k with y = Rs/r.  Scalar form (one sample).
__device__ __forceinline__ float tnfw_series_u(float u, float u2, const float4* t) {
  float p = fmaf(tnfw_coef(t, kFarTerms), u, tnfw_coef(t, kFarTerms - 1));
#pragma unroll
  for (int k = kFarTerms - 2; k >= 2; --k) p = fmaf(p, u, tnfw_coef(t, k));
  p = fmaf(p, u2, tnfw_coef(t, 0));
  return p * u2;
}

__device__ __forceinline__ float tnfw_series(float r2, const float4* t) {
  const float u = rsqrt_ftz(r2);
  return tnfw_series_u(u, u * u, t);
}

// The series truncated after d_K (K = 3 .. kFarTerms; K = kFarTerms is tnfw_series_u itself).
template <int K>
__device__ __forceinline__ float tnfw_series_k(float u, float u2, const float4* t) {
  static_assert(K >= 3 && K <= kFarTerms, "series length");
  float p = fmaf(tnfw_coef(t, K), u, tnfw_coef(t, K - 1));
#pragma unroll
  for (int k = K - 2; k >= 2; --k) p = fmaf(p, u, tnfw_coef(t, k));
  p = fmaf(p, u2, tnfw_coef(t, 0));
  return p * u2;
}

// Packed forms (two samples per instruction): element-wise the same operations, hence the same
// rounding, as the scalar forms.
__device__ __forceinline__ float2 tnfw_series2_u(float2 u, float2 u2, const float4* t) {
  float2 p = __ffma2_rn(tnfw_coef2(t, kFarTerms), u, tnfw_coef2(t, kFarTerms - 1));
#pragma unroll
  for (int k = kFarTerms - 2; k >= 2; --k) p = __ffma2_rn(p, u, tnfw_coef2(t, k));
  p = __ffma2_rn(p, u2, tnfw_coef2(t, 0));
  return __fmul2_rn(p, u2);
}

__device__ __forceinline__ float2 tnfw_series2(float2 r2, const float4* t) {
  const float2 u = make_float2(rsqrt_ftz(r2.x), rsqrt_ftz(r2.y));
  return tnfw_series2_u(u, __fmul2_rn(u, u), t);
}

template <int K>
__device__ __forceinline__ float2 tnfw_series2_k(float2 u, float2 u2, const float4* t) {
  static_assert(K >= 3 && K <= kFarTerms, "series length");
  float2 p = __ffma2_rn(tnfw_coef2(t, K), u, tnfw_coef2(t, K - 1));
#pragma unroll
  for (int k = K - 2; k >= 2; --k) p = __ffma2_rn(p, u, tnfw_coef2(t, k));
  p = __ffma2_rn(p, u2, tnfw_coef2(t, 0));
  return __fmul2_rn(p, u2);
}

// Annulus polynomial: A g = u^2 sum_j e_j t^j, t = a_t u + b_t (Horner in t).
__device__ __forceinline__ float tnfw_mid_u(float u, float u2, const float4* t, const float4* m) {
  const float x = fmaf(t[6].x, u, t[6].y);
  float p = fmaf(m[2].w, x, m[2].z);
  p = fmaf(p, x, m[2].y);
  p = fmaf(p, x, m[2].x);
  p = fmaf(p, x, m[1].w);
  p = fmaf(p, x, m[1].z);
  p = fmaf(p, x, m[1].y);
  p = fmaf(p, x, m[1].x);
  p = fmaf(p, x, m[0].w);
  p = fmaf(p, x, m[0].z);
  p = fmaf(p, x, m[0].y);
  p = fmaf(p, x, m[0].x);
  return p * u2;
}

__device__ __forceinline__ float2 tnfw_mid2_u(float2 u, float2 u2, const float4* t, const float4* m) {
  auto d = [](float v) { return make_float2(v, v); };
  const float2 x = __ffma2_rn(d(t[6].x), u, d(t[6].y));
  float2 p = __ffma2_rn(d(m[2].w), x, d(m[2].z));
  p = __ffma2_rn(p, x, d(m[2].y));
  p = __ffma2_rn(p, x, d(m[2].x));
  p = __ffma2_rn(p, x, d(m[1].w));
  p = __ffma2_rn(p, x, d(m[1].z));
  p = __ffma2_rn(p, x, d(m[1].y));
  p = __ffma2_rn(p, x, d(m[1].x));
  p = __ffma2_rn(p, x, d(m[0].w));
  p = __ffma2_rn(p, x, d(m[0].z));
  p = __ffma2_rn(p, x, d(m[0].y));
  p = __ffma2_rn(p, x, d(m[0].x));
  return __fmul2_rn(p, u2);
}

// Inside the annulus or closer: the closed forms (x >= 4) or the small-x forms (x < 4), times A.
// The x floor of 1e-6 (x^2 >= 1e-12) makes alpha vanish continuously at the subhalo centre.
static __device__ __noinline__ float tnfw_g_inner(float x2, float tau, float A, float C) {
  x2 = fmaxf(x2, 1e-12f);
  const float t2 = tau * tau, t2m1 = t2 - 1.f;
  return A * ((x2 >= 16.f) ? tnfw_g_far(x2, tau, t2, t2m1, C) : tnfw_g_near(x2, tau, t2, t2m1, C));
}

// A g for one pair at squared distance r2, any distance: the series beyond r_far, the annulus
// polynomial on [r_in, r_far) when the annulus block m is given, the closed forms inside.
__device__ __forceinline__ float tnfw_ag(float r2, const float4* t, const float4* m) {
  if (r2 >= t[1].x) return tnfw_series(r2, t);
  if (m != nullptr && r2 >= t[6].z) {
    const float u = rsqrt_ftz(r2);
    return tnfw_mid_u(u, u * u, t, m);
  }
  return tnfw_g_inner(r2 * t[1].y, t[1].z, t[1].w, t[6].w);
}

// One point-subhalo pair accumulated into (ax, ay); t is the subhalo's record, m its annulus
// block (or nullptr: closed forms inside r_far).
__device__ __forceinline__ void tnfw_pair(float px, float py, const float4* t, const float4* m, float& ax,
                                          float& ay) {
  const float dx = px + t[0].x, dy = py + t[0].z;
  const float k = tnfw_ag(fmaf(dx, dx, dy * dy), t, m);
  ax = fmaf(k, dx, ax);
  ay = fmaf(k, dy, ay);
}

// Writes subhalo j's record and annulus block into a table of n subhalos.  Not inlined, so
// that every prep kernel (one system, batched) runs the very same code and tables built by
// different launch paths are bitwise identical.
static __device__ __noinline__ void tnfw_write_table(float cx, float cy, float Rs, float alphaRs, float rt, int j,
                                                 int n, float4* __restrict__ tab) {
  float4 t[kSubStride], m[kMidStride];
  tnfw_constants(cx, cy, Rs, alphaRs, rt, t);
  tnfw_mid_constants(Rs, t, m);
  float4* o = tab + (size_t)kSubStride * j;
#pragma unroll
  for (int c = 0; c < kSubStride; ++c) o[c] = t[c];
  float4* om = tab + (size_t)kSubStride * n + (size_t)kMidStride * j;
#pragma unroll
  for (int c = 0; c < kMidStride; ++c) om[c] = m[c];
  static_assert(kFarTerms == 6, "the compact block holds d_0, d_2 .. d_6");
  float4* of = tab + (size_t)(kSubStride + kMidStride) * n + (size_t)kFarStride * j;
  of[0] = make_float4(t[0].x, t[0].z, t[1].x, t[5].x);
  of[1] = make_float4(t[5].y, t[2].x, t[2].z, t[3].x);
  of[2] = make_float4(t[3].z, t[4].x, t[4].z, 0.f);
}

__device__ __forceinline__ void alpha_nfw(float x, float y, float Rs, float alphaRs, float cx, float cy,
                                          float& ax, float& ay) {
  float dx = x - cx, dy = y - cy;
  float x2 = fmaxf((dx * dx + dy * dy) / (Rs * Rs), 1e-12f);
  float k = alphaRs / (kOneMinusLn2 * Rs) * nfw_h_over_x2(x2);
  ax = k * dx;
  ay = k * dy;
}

__device__ __forceinline__ void alpha_tnfw(float x, float y, float Rs, float alphaRs, float rt, float cx,
                                           float cy, float& ax, float& ay) {
  float4 t[kSubStride];
  tnfw_constants(cx, cy, Rs, alphaRs, rt, t);
  ax = 0.f; ay = 0.f;
  tnfw_pair(x, y, t, nullptr, ax, ay);
}

// Deflection of one deflector-list profile at (x, y); returns (ax, ay).
// Circular multipole of integer order m: kappa = r_E a_m cos(m (phi - phi_m)) / (2 r), alpha the
// gradient of its potential (r_E a_m r cos(m dphi) / (1 - m^2); (r_E a_1 / 2) r ln(r/r_E) cos(dphi)
// for m = 1), as radial and tangential components.  cos(m dphi), sin(m dphi) come from complex
// powers of e^(i dphi) = ((dx, dy)/r) e^(-i phi_m), so no arctangent is needed.
__device__ __forceinline__ void alpha_multipole(float x, float y, int m, float am, float phim, float cx, float cy,
                                                float rE, float& ax, float& ay) {
  const float dx = x - cx, dy = y - cy;
  const float r2 = dx * dx + dy * dy;
  if (!(r2 > 1e-40f)) { ax = 0.f; ay = 0.f; return; }
  const float inv = rsqrtf(r2), r = r2 * inv;
  const float c1 = dx * inv, s1 = dy * inv;
  float sm, cm;
  sincosf(phim, &sm, &cm);
  const float cd = c1 * cm + s1 * sm, sd = s1 * cm - c1 * sm;
  float ar, at;
  if (m == 1) {
    const float B = 0.5f * rE * am;
    const float L = logf(r / rE);
    ar = B * (L + 1.f) * cd;
    at = -B * L * sd;
  } else {
    float cmd = cd, smd = sd;
    for (int k = 1; k < m; ++k) {
      const float c2 = cmd * cd - smd * sd;
      smd = smd * cd + cmd * sd;
      cmd = c2;
    }
    const float A = rE * am / (1.f - (float)(m * m));
    ar = A * cmd;
    at = -A * (float)m * smd;
  }
  ax = ar * c1 - at * s1;
  ay = ar * s1 + at * c1;
}

// Cored steep ellipsoid, kappa = A / (2 (s^2 + x'^2 + y'^2/q^2)^(3/2)) in the frame of phi.
// Closed form: kappa is -(A/s) d/ds of the softened isothermal ellipsoid's 1/(2 sqrt(s^2 + xi^2)),
// so alpha is -(A/s) d/ds of its deflection; with psi = sqrt(q^2 (s^2 + x'^2) + y'^2) and
// D = (1 + q^2) s^2 + 2 s psi + x'^2 + y'^2 (all terms positive, no cancellation):
//   alpha'_x = A q x' (psi + q^2 s) / (s psi D),  alpha'_y = A q y' (psi + s) / (s psi D).
__device__ __forceinline__ void alpha_cse(float x, float y, float A, float s, float q, float phi, float cx, float cy,
                                          float& ax, float& ay) {
  float sp, cp;
  sincosf(phi, &sp, &cp);
  const float dx = x - cx, dy = y - cy;
  const float xp = cp * dx + sp * dy, yp = -sp * dx + cp * dy;
  const float q2 = q * q;
  const float psi = sqrtf(q2 * (s * s + xp * xp) + yp * yp);
  const float D = (1.f + q2) * s * s + 2.f * s * psi + xp * xp + yp * yp;
  const float f = A * q / (s * psi * D);
  const float axp = f * xp * (psi + q2 * s), ayp = f * yp * (psi + s);
  ax = cp * axp - sp * ayp;
  ay = sp * axp + cp * ayp;
}

// Elliptical profile given as a sum of CSEs in units of Rs (tables of cse_fits.h):
//   kappa = norm sum_i a_i / (2 (sigma_i^2 + xi^2/Rs^2)^(3/2)),  xi^2 = q x'^2 + y'^2/q.
// In the CSE frame xi_c^2 = xi^2/q each term is a CSE with s_i = sigma_i Rs/sqrt(q) and
// A_i = norm a_i Rs^3 q^(-3/2), hence A_i q / s_i = norm a_i Rs^2 / sigma_i.  All terms add with
// the same sign (a_i >= 0), so the FP32 sum has no cancellation.
__device__ __forceinline__ void alpha_cse_sum(const float* sig, const float* amp, float norm, float Rs, float q,
                                              float phi, float cx, float cy, float x, float y, float& ax,
                                              float& ay) {
  float sp, cp;
  sincosf(phi, &sp, &cp);
  const float dx = x - cx, dy = y - cy;
  const float xp = cp * dx + sp * dy, yp = -sp * dx + cp * dy;
  const float q2 = q * q, isq = rsqrtf(q), xx = xp * xp, yy = yp * yp, r2 = xx + yy;
  const float nR2 = norm * Rs * Rs;
  float axp = 0.f, ayp = 0.f;
  for (int i = 0; i < kCseTerms; ++i) {
    const float s = sig[i] * Rs * isq;
    const float psi = sqrtf(q2 * (s * s + xx) + yy);
    const float D = (1.f + q2) * s * s + 2.f * s * psi + r2;
    const float f = nR2 * amp[i] / (sig[i] * psi * D);
    axp = fmaf(f, psi + q2 * s, axp);
    ayp = fmaf(f, psi + s, ayp);
  }
  axp *= xp;
  ayp *= yp;
  ax = cp * axp - sp * ayp;
  ay = sp * axp + cp * ayp;
}

// Elliptical multipole (m, a_m, phi_m, q, phi_e, cx, cy, r_E).  2 kappa r depends on the polar
// angle theta alone; with its Fourier coefficients c_k (scaled by a_m r_E, computed on the host
// once per system) the potential is psi = r F(theta) + (1/2) r ln(r/r_E) h_1(theta), where
// F = sum over k != +-1 of c_k e^{ik theta} / (1 - k^2) and h_1 = 2 Re(c_1 e^{i theta}) is the
// k = +-1 part (present for odd m), whose r ln r potential has Laplacian h_1/r.  alpha = grad psi
// from the radial derivative (F + (L + 1) h_1/2) and the tangential one (F' + L h_1'/2), L = ln(r/r_E).
__device__ __forceinline__ void alpha_multipole_ell(const float* p, const float* c, int K, float x, float y,
                                                    float& ax, float& ay) {
  float se, ce;
  sincosf(p[4], &se, &ce);
  const float dx = x - p[5], dy = y - p[6];
  const float xp = ce * dx + se * dy, yp = -se * dx + ce * dy;
  const float r2 = xp * xp + yp * yp;
  if (r2 < 1e-24f) { ax = 0.f; ay = 0.f; return; }
  const float ir = rsqrtf(r2), r = r2 * ir;
  const float ct = xp * ir, st = yp * ir;
  float F = c[0], Fd = 0.f;
  float zr = ct, zi = st;  // e^{i k theta}
  for (int k = 2; k <= K; ++k) {
    const float nr = zr * ct - zi * st, ni = zr * st + zi * ct;
    zr = nr;
    zi = ni;
    // (ct, st) is a unit vector only to FP32 rounding, and its k-th power drifts in magnitude
    // by about k/2 of that (1e-5 at the 300th harmonic): every fourth power is scaled back to
    // unit magnitude, 1/|z| ~ 1.5 - |z|^2 / 2 to second order
    if ((k & 3) == 0) {
      const float g = fmaf(-0.5f, fmaf(zr, zr, zi * zi), 1.5f);
      zr *= g;
      zi *= g;
    }
    const float w = 2.f / (1.f - (float)(k * k));
    const float pr = c[2 * k] * zr - c[2 * k + 1] * zi, pim = c[2 * k] * zi + c[2 * k + 1] * zr;
    F = fmaf(w, pr, F);
    Fd = fmaf(-w * (float)k, pim, Fd);
  }
  const float A = 2.f * c[2], B = -2.f * c[3];
  const float h1 = A * ct + B * st, h1d = B * ct - A * st;
  const float L = logf(r / p[7]);
  const float ar = F + 0.5f * (L + 1.f) * h1, at = Fd + 0.5f * L * h1d;
  const float axp = ar * ct - at * st, ayp = ar * st + at * ct;
  ax = ce * axp - se * ayp;
  ay = se * axp + ce * ayp;
}

// One deflector at (x, y); ell_c / ell_K: the system's elliptical-multipole coefficients.
static __device__ __noinline__ void alpha_profile(const DevProfile& P, const float* ell_c, int ell_K, float x, float y,
                                                  float& ax, float& ay) {
  const float* p = P.p;
  switch (P.type) {
    case LENS_MULTIPOLE_ELL: alpha_multipole_ell(p, ell_c, ell_K, x, y, ax, ay); return;
    case LENS_SIS: alpha_sis(x, y, p[0], p[1], p[2], ax, ay); return;
    case LENS_SIE: alpha_sie(x, y, p[0], p[1], p[2], p[3], p[4], ax, ay); return;
    case LENS_EPL: alpha_epl(x, y, p[0], p[1], p[2], p[3], p[4], p[5], ax, ay); return;
    case LENS_SHEAR: ax = p[0] * x + p[1] * y; ay = p[1] * x - p[0] * y; return;
    case LENS_POINT_MASS: alpha_point_mass(x, y, p[0], p[1], p[2], ax, ay); return;
    case LENS_NFW: alpha_nfw(x, y, p[0], p[1], p[2], p[3], ax, ay); return;
    case LENS_TNFW: alpha_tnfw(x, y, p[0], p[1], p[2], p[3], p[4], ax, ay); return;
    case LENS_EPL_E1E2: {
      float q, phi;
      e1e2_to_qphi(p[2], p[3], q, phi);
      alpha_epl(x, y, p[0], p[1], q, phi, p[4], p[5], ax, ay);
      return;
    }
    case LENS_SIE_E1E2: {
      float q, phi;
      e1e2_to_qphi(p[1], p[2], q, phi);
      alpha_sie(x, y, p[0], q, phi, p[3], p[4], ax, ay);
      return;
    }
    case LENS_CSE: {
      float q, phi;
      e1e2_to_qphi(p[2], p[3], q, phi);
      alpha_cse(x, y, p[0], p[1], q, phi, p[4], p[5], ax, ay);
      return;
    }
    case LENS_NFW_ELLIPSE_CSE: {
      float q, phi;
      e1e2_to_qphi(p[2], p[3], q, phi);
      alpha_cse_sum(kCseNfwSigma, kCseNfwAmp, p[1] / (kOneMinusLn2 * 4.f * p[0]), p[0], q, phi, p[4], p[5], x, y, ax,
                    ay);
      return;
    }
    case LENS_HERNQUIST_ELLIPSE_CSE: {
      float q, phi;
      e1e2_to_qphi(p[2], p[3], q, phi);
      alpha_cse_sum(kCseHernquistSigma, kCseHernquistAmp, p[0], p[1], q, phi, p[4], p[5], x, y, ax, ay);
      return;
    }
    case LENS_MULTIPOLE: alpha_multipole(x, y, __float2int_rn(p[0]), p[1], p[2], p[3], p[4], p[5], ax, ay); return;
    case LENS_EPL_MULTIPOLE_M1M3M4: {
      float q, phi;
      e1e2_to_qphi(p[2], p[3], q, phi);
      alpha_epl(x, y, p[0], p[1], q, phi, p[4], p[5], ax, ay);
      const int ms[3] = {1, 3, 4};
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        float mx, my;
        alpha_multipole(x, y, ms[i], p[6 + 2 * i], phi + p[7 + 2 * i], p[4], p[5], p[0], mx, my);
        ax += mx;
        ay += my;
      }
      return;
    }
    default: ax = 0.f; ay = 0.f; return;
  }
}

// ---------------------------------------------------------------------------- Sersic source
// Elliptical Sersic: the profile's point-independent quantities and its value at a point.
struct SersicFrame {
  float amp, Rs, n, q, cp, sp, bn, cx, cy;
};

__device__ __forceinline__ SersicFrame sersic_frame(float amp, float Rs, float n, float q, float phi, float cx,
                                                    float cy) {
  SersicFrame f;
  sincosf(phi, &f.sp, &f.cp);
  f.amp = amp;
  f.Rs = Rs;
  f.n = n;
  f.q = q;
  f.bn = 1.9992f * n - 0.3271f;
  f.cx = cx;
  f.cy = cy;
  return f;
}

__device__ __forceinline__ float sersic_at(float x, float y, const SersicFrame& f) {
  float xp, yp;
  to_frame(x - f.cx, y - f.cy, f.cp, f.sp, xp, yp);
  float R = sqrtf(f.q * xp * xp + yp * yp / f.q);
  float pw = exp2f(log2f(R / f.Rs) / f.n);
  return f.amp * expf(-f.bn * (pw - 1.f));
}

__device__ __forceinline__ float sersic(float x, float y, float amp, float Rs, float n, float q, float phi,
                                        float cx, float cy) {
  return sersic_at(x, y, sersic_frame(amp, Rs, n, q, phi, cx, cy));
}

// Cartesian shapelets: the orthonormal Hermite functions phi_n(u) by their normalised
// three-term recurrence phi_(n+1) = sqrt(2/(n+1)) u phi_n - sqrt(n/(n+1)) phi_(n-1),
// phi_0 = pi^(-1/4) exp(-u^2/2), then I = sum_k amp_k phi_n1(u) phi_n2(v) / beta in the
// amplitude order n = n1 + n2 ascending, n1 descending.
__device__ __forceinline__ float shapelets(const float* p, const float* coef, float x, float y) {
  constexpr int N = LENS_MAX_SHAPELET_NMAX;
  const int nmax = __float2int_rn(p[0]);
  const float ib = 1.f / p[1];
  const float u = (x - p[2]) * ib, v = (y - p[3]) * ib;
  float fu[N + 1], fv[N + 1];
  fu[0] = 0.75112554446494248f * expf(-0.5f * u * u);
  fv[0] = 0.75112554446494248f * expf(-0.5f * v * v);
  fu[1] = 1.41421356237309505f * u * fu[0];
  fv[1] = 1.41421356237309505f * v * fv[0];
#pragma unroll
  for (int n = 1; n < N; ++n) {
    const float a = sqrtf(2.f / (n + 1)), b = sqrtf((float)n / (n + 1));
    fu[n + 1] = a * u * fu[n] - b * fu[n - 1];
    fv[n + 1] = a * v * fv[n] - b * fv[n - 1];
  }
  float sum = 0.f;
#pragma unroll
  for (int n = 0; n <= N; ++n) {
    if (n > nmax) break;
#pragma unroll
    for (int n1 = n; n1 >= 0; --n1) sum = fmaf(coef[n * (n + 1) / 2 + (n - n1)], fu[n1] * fv[n - n1], sum);
  }
  return sum * ib;
}

static __device__ __noinline__ float source_light(int type, const float* p, const float* coef, float x, float y) {
  switch (type) {
    case LIGHT_SHAPELETS: return shapelets(p, coef, x, y);
    case LIGHT_SERSIC_ELLIPSE_Q_PHI: return sersic(x, y, p[0], p[1], p[2], p[3], p[4], p[5], p[6]);
    case LIGHT_SERSIC_ELLIPSE: {
      float q, phi;
      e1e2_to_qphi(p[3], p[4], q, phi);
      return sersic(x, y, p[0], p[1], p[2], q, phi, p[5], p[6]);
    }
    case LIGHT_SERSIC: return sersic(x, y, p[0], p[1], p[2], 1.f, 0.f, p[3], p[4]);
    default: return 0.f;
  }
}

// Grid coordinate of column j (or row i), sub-sample b of s: centre-relative offsets in pixels.
__device__ __forceinline__ float grid_coord(float c0, int j, int n, int b, int s, float dpix) {
  return c0 + ((float)j - 0.5f * (float)(n - 1) + ((float)b + 0.5f) / (float)s - 0.5f) * dpix;
}

}  // namespace ls

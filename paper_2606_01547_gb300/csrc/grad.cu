// Chi^2 log-likelihood and its hand-written adjoint (the gradient-based fitting of the paper's
// lens-modelling section), batched over parameter points.
//
// Forward, per parameter point p (15 parameters: EPL_E1E2 6, SHEAR 2, SERSIC_ELLIPSE 7):
//   m0 = dpix^2/s^2 sum_samples I(theta - alpha_EPL - alpha_shear - alpha_sub)   (alpha_sub fixed)
//   m  = K (*) m0                                                     (PSF convolution)
//   logL = -1/2 sum_pix (d - m)^2 / sigma^2,   sigma^2 = sigma_bkg^2 + max(m, 0)/t_exp
// Reverse accumulation:
//   g_m  = dlogL/dm = r/sigma^2 + 1/2 r^2/sigma^4 [m > 0]/t_exp,  r = d - m
//   g_m0 = K^T g_m                                                    (PSF transpose = correlation)
//   g_I  = g_m0 dpix^2/s^2 at each sample of the pixel                 (bin-down spread)
//   dlogL/dp_src  = sum g_I dI/dp_src
//   dlogL/dp_lens = sum g_I (-dI/dbeta . dalpha/dp_lens)               (lens equation)
// The per-sample local Jacobians dalpha_EPL/dp and dI/d(p_src, beta) are closed forms (the EPL's
// q and t derivatives as tangent recurrences beside its series); every reduction is a
// fixed-order two-stage tree (deterministic).
#include <algorithm>

#include "kernels.h"
#include "lens_sim.h"
#include "sim_internal.h"

namespace ls {

constexpr int kGradThreads = 256;
// Samples (pixels in the forward model) per thread of the per-point kernels: each block fills
// its EPL table and reduces its partial sums once, so a few samples per thread amortise that.
constexpr int kWorkPerThread = 4;
inline int blocks_per_point(long long n_work) {
  return (int)std::max<long long>(1, std::min<long long>((n_work + kGradThreads * kWorkPerThread - 1) /
                                                            (kGradThreads * kWorkPerThread), 64));
}
// A value and its derivatives along 6 parameters (the per-sample local Jacobians).
struct Jac6 {
  float v;
  float d[6];
};

__device__ __forceinline__ Jac6 jac_const(float v) {
  Jac6 r;
  r.v = v;
#pragma unroll
  for (int i = 0; i < 6; ++i) r.d[i] = 0.f;
  return r;
}

// Per parameter point, the EPL series coefficients c_n (the division alpha_epl makes) and
// dc_n/dt = 4n/(2n + 2 - t)^2 for n = 1..kEplTab: t = gamma - 1 is the same for every sample of
// a point, so each block fills the table once in shared memory instead of dividing per term and
// sample.  kEplTab covers the longest series (epl_terms <= 200; the adjoint's own count is
// capped at kEplTab).
constexpr int kEplTab = 256;
__device__ __forceinline__ void fill_epl_table(const float* P, float2* tab) {
  const float t = P[1] - 1.f;
  for (int n = threadIdx.x + 1; n <= kEplTab; n += blockDim.x) {
    const float inv = 1.f / ((2.f * n + 2.f) - t);
    tab[n - 1] = make_float2(epl_coef(n, t), 4.f * n * inv * inv);
  }
}

// Per parameter point: the lens and source frames and the adjoint's chain-rule factors, the
// same for every sample of the point, so each block computes them once in shared memory.
struct PointFrame {
  EplFrame lens;
  SersicFrame src;
  float l_qc, l_pc;  // lens e1, e2 -> (q, phi): (dq/dc)/c and 1/(2 c^2), c = |e|
  float l_gq;        // -df/dq = 2/(1 + q)^2
  float l_dT;        // t / theta_E
  float l_k0;        // t/(2q) - 1/(1 + q), the point-independent part of d ln(prefactor)/dq
  float s_qc, s_pc;  // the same for the source ellipticity
  float s_in;        // 1/n
  int nt_adj;        // series terms of the adjoint: the value's own count (|Omega_n| <= f^n
                     // below 2^-26, as in the image kernels) plus the terms that bring the
                     // tangents' n f^(n-1) below the same bound
};

__device__ __forceinline__ void point_frame(const float* P, PointFrame& F) {
  float q, phi;
  e1e2_to_qphi(P[2], P[3], q, phi);
  F.lens = epl_frame(P[0], P[1], q, phi);
  const float lc = sqrtf(P[2] * P[2] + P[3] * P[3]);
  F.l_qc = -2.f / ((1.f + lc) * (1.f + lc)) / lc;
  F.l_pc = 0.5f / (lc * lc);
  F.l_gq = 2.f / ((1.f + q) * (1.f + q));
  F.l_dT = F.lens.t / P[0];
  F.l_k0 = F.lens.t / (2.f * q) - 1.f / (1.f + q);
  const float f = F.lens.f;
  // The adjoint's value series is summed at least as far as the image kernels' (tail below
  // 2^-26 of the sum), so its traced positions are those of the forward model to FP32
  // resolution, and its tangent series to the same bound.
  const int nv = F.lens.nt;
  F.nt_adj = nv == 0 ? 0 : min(nv + (int)ceilf(logf((float)nv) / -logf(f)) + 1, kEplTab);
  float qs, phis;
  e1e2_to_qphi(P[11], P[12], qs, phis);
  F.src = sersic_frame(P[8], P[9], P[10], qs, phis, P[13], P[14]);
  const float sc = sqrtf(P[11] * P[11] + P[12] * P[12]);
  F.s_qc = -2.f / ((1.f + sc) * (1.f + sc)) / sc;
  F.s_pc = 0.5f / (sc * sc);
  F.s_in = 1.f / P[10];
}

// ---------------------------------------------------------------------------- sample geometry
__device__ __forceinline__ void sample_coords(const DevSystem& g, long long idx, float& x, float& y, int& pix) {
  const int s = g.s;
  const int b = (int)(idx % s);
  long long t = idx / s;
  const int a = (int)(t % s);
  t /= s;
  const int j = (int)(t % g.nx);
  const int i = (int)(t / g.nx);
  x = grid_coord(g.x0, j, g.nx, b, s, g.dpix);
  y = grid_coord(g.y0, i, g.ny, a, s, g.dpix);
  pix = i * g.nx + j;
}

// ---------------------------------------------------------------------------- forward model
__device__ __forceinline__ float model_sample(float x, float y, float2 asub, const float* __restrict__ P,
                                              const PointFrame& F, const float2* __restrict__ tab) {
  float ex, ey;
  alpha_epl_at(x, y, F.lens, P[4], P[5], [tab](int n) { return tab[n - 1].x; }, ex, ey);
  const float bx = x - ex - (P[6] * x + P[7] * y) - asub.x;
  const float by = y - ey - (P[7] * x - P[6] * y) - asub.y;
  return sersic_at(bx, by, F.src);
}

__global__ void __launch_bounds__(kGradThreads) forward_model_kernel(const __grid_constant__ DevSystem g,
                                                                     const float* __restrict__ params,
                                                                     const float2* __restrict__ asub,
                                                                     float* __restrict__ m0, int unit_amp) {
  __shared__ float P[LENS_N_FREE_PARAMS];
  __shared__ float2 tab[kEplTab];
  __shared__ PointFrame F;
  const int p = blockIdx.y;
  if (threadIdx.x < LENS_N_FREE_PARAMS) P[threadIdx.x] = params[p * LENS_N_FREE_PARAMS + threadIdx.x];
  if (unit_amp && threadIdx.x == 8) P[8] = 1.f;  // linear solve: the model per unit source amplitude
  __syncthreads();
  fill_epl_table(P, tab);
  if (threadIdx.x == 0) point_frame(P, F);
  __syncthreads();
  const int npix = g.nx * g.ny;
  const int s2 = g.s * g.s;
  for (int pix = blockIdx.x * blockDim.x + threadIdx.x; pix < npix; pix += gridDim.x * blockDim.x) {
    float acc = 0.f;
    for (int k = 0; k < s2; ++k) {
      const long long idx = (long long)pix * s2 + k;
      float x, y;
      int pp;
      sample_coords(g, idx, x, y, pp);
      acc += model_sample(x, y, asub[idx], P, F, tab);
    }
    m0[(size_t)p * npix + pix] = acc * (g.dpix * g.dpix / (float)s2);
  }
}

// ---------------------------------------------------------------------------- block reduction
template <int W>
__device__ __forceinline__ void block_reduce_store(float (&v)[W], float* __restrict__ dst) {
  __shared__ float red[kGradThreads / 32][W];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < W; ++c) {
    float x = v[c];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
    if (lane == 0) red[w][c] = x;
  }
  __syncthreads();
  if (threadIdx.x < W) {
    float x = 0.f;
#pragma unroll
    for (int ww = 0; ww < kGradThreads / 32; ++ww) x += red[ww][threadIdx.x];
    dst[threadIdx.x] = x;
  }
}

// Per-pixel chi^2 terms and dlogL/dm; partial sums of (d-m)^2/sigma^2 per block.
__global__ void __launch_bounds__(kGradThreads) likelihood_kernel(const float* __restrict__ m,
                                                                  const float* __restrict__ d, int npix,
                                                                  float var_bkg, float inv_t,
                                                                  float* __restrict__ gm,
                                                                  float* __restrict__ partial, int nblk) {
  const int p = blockIdx.y;
  const int pix = blockIdx.x * blockDim.x + threadIdx.x;
  float v[1] = {0.f};
  if (pix < npix) {
    const float mv = m[(size_t)p * npix + pix];
    const float pos = mv > 0.f ? 1.f : 0.f;
    const float var = var_bkg + pos * mv * inv_t;
    const float r = d[pix] - mv;
    const float iv = 1.f / var;
    v[0] = r * r * iv;
    if (gm) gm[(size_t)p * npix + pix] = r * iv + 0.5f * r * r * iv * iv * pos * inv_t;
  }
  block_reduce_store<1>(v, partial + (size_t)p * nblk + blockIdx.x);
}

// out[p * width + c] = scale * sum_b partial[(p * nblk + b) * width + c], fixed order.
__global__ void reduce_partials_kernel(const float* __restrict__ partial, int nblk, int width, float scale,
                                       float* __restrict__ out, int n_points) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_points * width) return;
  const int p = t / width, c = t - p * width;
  float acc = 0.f;
  for (int b = 0; b < nblk; ++b) acc += partial[((size_t)p * nblk + b) * width + c];
  out[t] = scale * acc;
}

// ---------------------------------------------------------------------------- local Jacobians
// EPL deflection with tangents along (theta_E, gamma, e1, e2, cx, cy) at a fixed point.  The
// value is the series of alpha_epl (Tessore & Metcalf 2015); of the tangents only d/dq and d/dt
// run through the series (two complex tangent recurrences beside it), the rest are closed forms:
//   theta_E: alpha is proportional to b^t with b = theta_E sqrt(q), so d alpha = t alpha / theta_E;
//   cx, cy:  minus the Hessian A of the potential; its trace is 2 kappa with
//            kappa = (2 - t)/2 (b/R)^t, and its shear follows from Euler's relation
//            x'.grad alpha' = (1 - t) alpha' of a deflection homogeneous of degree 1 - t;
//   phi:     the frame rotation, d alpha'/dphi = J alpha' - A J x' with J the quarter turn;
//   e1, e2:  chain rule through q = (1 - c)/(1 + c), c = |e|, phi = atan2(e2, e1)/2.
__device__ __forceinline__ void epl_alpha_jac(float x, float y, const float* __restrict__ P, const PointFrame& F,
                                              const float2* __restrict__ tab, Jac6& ax, Jac6& ay) {
  const float t = F.lens.t, e1 = P[2], e2 = P[3];
  const float q = F.lens.q, cp = F.lens.cp, sp = F.lens.sp;
  const float dx = x - P[4], dy = y - P[5];
  const float xp = cp * dx + sp * dy, yp = -sp * dx + cp * dy;
  const float R = sqrtf(q * q * xp * xp + yp * yp);
  if (R < 1e-12f) { ax = jac_const(0.f); ay = jac_const(0.f); return; }
  const float iR = 1.f / R;
  const float b = F.lens.b, f = F.lens.f;
  const float er = q * xp * iR, ei = yp * iR;        // e = (q x' + i y') / R
  const float e2r = er * er - ei * ei, e2i = 2.f * er * ei;
  const float zr = -f * e2r, zi = -f * e2i;          // Z = -f e^2
  const float Rq = q * xp * xp * iR;                 // dR/dq
  const float eqr = (xp - er * Rq) * iR, eqi = -ei * Rq * iR;  // de/dq
  const float gq = F.l_gq;                           // -df/dq
  const float zqr = gq * e2r - 2.f * f * (er * eqr - ei * eqi);  // dZ/dq = gq e^2 - 2 f e de/dq
  const float zqi = gq * e2i - 2.f * f * (er * eqi + ei * eqr);
  float omr = er, omi = ei, sr = er, si = ei;        // Omega_n and its sum
  float otr = 0.f, oti = 0.f, str = 0.f, sti = 0.f;  // d/dt
  float oqr = eqr, oqi = eqi, sqr = eqr, sqi = eqi;  // d/dq
  const int nt = F.nt_adj;
  for (int n = 1; n <= nt; ++n) {
    const float2 cc = tab[n - 1];
    const float cn = cc.x, cnt = cc.y;  // c_n, dc_n/dt
    const float zor = omr * zr - omi * zi, zoi = omr * zi + omi * zr;          // Z Omega_{n-1}
    const float nqr = cn * ((zqr * omr - zqi * omi) + (zr * oqr - zi * oqi));
    const float nqi = cn * ((zqr * omi + zqi * omr) + (zr * oqi + zi * oqr));
    const float ntr = cnt * zor + cn * (zr * otr - zi * oti);
    const float nti = cnt * zoi + cn * (zr * oti + zi * otr);
    omr = cn * zor;
    omi = cn * zoi;
    otr = ntr;
    oti = nti;
    oqr = nqr;
    oqi = nqi;
    sr += omr;
    si += omi;
    str += otr;
    sti += oti;
    sqr += oqr;
    sqi += oqi;
  }
  const float bR = b * iR, lbR = log2f(bR);
  const float pw = exp2f((t - 1.f) * lbR);           // (b/R)^(t-1)
  const float pref = F.lens.b2q * pw;
  const float apx = pref * sr, apy = pref * si;      // alpha' in the lens frame
  const float ln_bR = lbR * 0.693147180559945f;
  const float atx = apx * ln_bR + pref * str, aty = apy * ln_bR + pref * sti;
  const float dlnP = F.l_k0 + (1.f - t) * Rq * iR;
  const float aqx = pref * (dlnP * sr + sqr), aqy = pref * (dlnP * si + sqi);
  const float kap = 0.5f * (2.f - t) * pw * bR;
  const float U = (1.f - t) * apx - kap * xp, V = (1.f - t) * apy - kap * yp;
  const float ir2 = 1.f / (xp * xp + yp * yp);
  const float g1 = (U * xp - V * yp) * ir2, g2 = (U * yp + V * xp) * ir2;
  const float a11 = kap + g1, a22 = kap - g1, a12 = g2;
  const float afx = -apy - (a12 * xp - a11 * yp);    // J alpha' - A J x', J x' = (-y', x')
  const float afy = apx - (a22 * xp - a12 * yp);
  auto rot_x = [&](float vx, float vy) { return cp * vx - sp * vy; };
  auto rot_y = [&](float vx, float vy) { return sp * vx + cp * vy; };
  ax.v = rot_x(apx, apy);
  ay.v = rot_y(apx, apy);
  const float dT = F.l_dT;
  ax.d[0] = dT * ax.v;
  ay.d[0] = dT * ay.v;
  ax.d[1] = rot_x(atx, aty);
  ay.d[1] = rot_y(atx, aty);
  const float qx = rot_x(aqx, aqy), qy = rot_y(aqx, aqy), fx = rot_x(afx, afy), fy = rot_y(afx, afy);
  const float qc = F.l_qc, pc = F.l_pc;  // (dq/dc)/c, dphi/de scale
  ax.d[2] = qx * qc * e1 - fx * pc * e2;
  ay.d[2] = qy * qc * e1 - fy * pc * e2;
  ax.d[3] = qx * qc * e2 + fx * pc * e1;
  ay.d[3] = qy * qc * e2 + fy * pc * e1;
  // Hessian in the image frame: columns Rot A Rot^T e_x and Rot A Rot^T e_y; d/dc = -column
  const float hx1 = a11 * cp - a12 * sp, hx2 = a12 * cp - a22 * sp;   // A Rot^T e_x, Rot^T e_x = (cp, -sp)
  const float hy1 = a11 * sp + a12 * cp, hy2 = a12 * sp + a22 * cp;   // A Rot^T e_y, Rot^T e_y = (sp, cp)
  ax.d[4] = -rot_x(hx1, hx2);
  ay.d[4] = -rot_y(hx1, hx2);
  ax.d[5] = -rot_x(hy1, hy2);
  ay.d[5] = -rot_y(hy1, hy2);
}

// Sersic with tangents along (R_s, n, e1, e2, beta_x, beta_y), in closed form: with
// rho = R/R_s, w = rho^(1/n) and ln I = ln amp - b_n (w - 1),
//   d ln I/dR_s = b_n w / (n R_s),  d ln I/dn = -b_n' (w - 1) + b_n w ln(rho) / n^2,
//   d ln I/dR = -b_n w / (n R),
// and R = sqrt(q x'^2 + y'^2/q) differentiated along q, phi (dx'/dphi = y', dy'/dphi = -x'),
// beta_x and beta_y; e1, e2 -> (q, phi) by the chain rule.  dI/damp = I/amp and
// dI/dc = -dI/dbeta follow without tangents.
__device__ __forceinline__ Jac6 sersic_jac(float bx, float by, const float* __restrict__ P, const PointFrame& F) {
  const float Rs = P[9], e1 = P[11], e2 = P[12];
  const float q = F.src.q, cp = F.src.cp, sp = F.src.sp;
  const float dx = bx - P[13], dy = by - P[14];
  const float xp = cp * dx + sp * dy, yp = -sp * dx + cp * dy;
  const float R = sqrtf(q * xp * xp + yp * yp / q);
  const float bn = F.src.bn;
  Jac6 I;
  if (R <= 0.f) {  // rho^(1/n) = 0: I = amp e^(b_n), which depends on n only
    I = jac_const(P[8] * expf(bn));
    I.d[1] = 1.9992f * I.v;
    return I;
  }
  const float in = F.s_in, lr = log2f(R / Rs);
  const float w = exp2f(lr * in);
  I.v = P[8] * expf(-bn * (w - 1.f));
  const float bw = bn * w * in;
  const float dR = -bw / R;  // d ln I / dR
  I.d[0] = I.v * bw / Rs;
  I.d[1] = I.v * (bw * lr * 0.693147180559945f * in - 1.9992f * (w - 1.f));
  const float Rx = q * xp / R, Ry = yp / (q * R);          // dR/dx', dR/dy'
  const float Rq = (xp * xp - yp * yp / (q * q)) / (2.f * R);
  const float Rphi = Rx * yp - Ry * xp;
  const float qc = F.s_qc, pc = F.s_pc;
  I.d[2] = I.v * dR * (Rq * qc * e1 - Rphi * pc * e2);
  I.d[3] = I.v * dR * (Rq * qc * e2 + Rphi * pc * e1);
  I.d[4] = I.v * dR * (Rx * cp - Ry * sp);
  I.d[5] = I.v * dR * (Rx * sp + Ry * cp);
  return I;
}

// Three blocks per SM (24 warps): the series recurrences are latency-bound chains, and the
// extra warps hide more of that latency than the few spilled registers cost.
__global__ void __launch_bounds__(kGradThreads, 3) backward_kernel(const __grid_constant__ DevSystem g,
                                                                const float* __restrict__ params,
                                                                const float2* __restrict__ asub,
                                                                const float* __restrict__ gm0,
                                                                float* __restrict__ partial, int nblk) {
  __shared__ float P[LENS_N_FREE_PARAMS];
  __shared__ float2 tab[kEplTab];
  __shared__ PointFrame F;
  const int p = blockIdx.y;
  if (threadIdx.x < LENS_N_FREE_PARAMS) P[threadIdx.x] = params[p * LENS_N_FREE_PARAMS + threadIdx.x];
  __syncthreads();
  fill_epl_table(P, tab);
  if (threadIdx.x == 0) point_frame(P, F);
  __syncthreads();
  const int npix = g.nx * g.ny;
  const int s2 = g.s * g.s;
  const long long n_samples = (long long)npix * s2;
  const float w = g.dpix * g.dpix / (float)s2;
  float acc[LENS_N_FREE_PARAMS];
#pragma unroll
  for (int c = 0; c < LENS_N_FREE_PARAMS; ++c) acc[c] = 0.f;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n_samples;
       idx += (long long)nblk * blockDim.x) {
    float x, y;
    int pix;
    sample_coords(g, idx, x, y, pix);
    const float gI = gm0[(size_t)p * npix + pix] * w;
    Jac6 ax, ay;
    epl_alpha_jac(x, y, P, F, tab, ax, ay);
    const float2 as = asub[idx];
    const float bx = x - ax.v - (P[6] * x + P[7] * y) - as.x;
    const float by = y - ay.v - (P[7] * x - P[6] * y) - as.y;
    const Jac6 I = sersic_jac(bx, by, P, F);
    const float dIdbx = I.d[4], dIdby = I.d[5];
    // lens parameters: beta = theta - alpha  ->  dI/dp = -(dI/dbx dax/dp + dI/dby day/dp)
#pragma unroll
    for (int c = 0; c < 6; ++c) acc[c] -= gI * (dIdbx * ax.d[c] + dIdby * ay.d[c]);
    // shear: alpha = (g1 x + g2 y, g2 x - g1 y)
    acc[6] -= gI * (dIdbx * x - dIdby * y);
    acc[7] -= gI * (dIdbx * y + dIdby * x);
    // source parameters
    acc[8] += gI * (I.v / P[8]);
    acc[9] += gI * I.d[0];
    acc[10] += gI * I.d[1];
    acc[11] += gI * I.d[2];
    acc[12] += gI * I.d[3];
    acc[13] -= gI * dIdbx;
    acc[14] -= gI * dIdby;
  }
  block_reduce_store<LENS_N_FREE_PARAMS>(acc, partial + ((size_t)p * nblk + blockIdx.x) * LENS_N_FREE_PARAMS);
}

// Linear amplitude solve: with data-based weights w = 1/(sigma_bkg^2 + max(d,0)/t_exp), the
// weighted sums A = sum w d m1, B = sum w m1^2, C = sum w d^2 of the unit-amplitude model m1.
__global__ void __launch_bounds__(kGradThreads) normal_eq_kernel(const float* __restrict__ m1,
                                                                 const float* __restrict__ d, int npix,
                                                                 float var_bkg, float inv_t,
                                                                 float* __restrict__ partial, int nblk) {
  const int p = blockIdx.y;
  const int pix = blockIdx.x * blockDim.x + threadIdx.x;
  float v[3] = {0.f, 0.f, 0.f};
  if (pix < npix) {
    const float dv = d[pix], mv = m1[(size_t)p * npix + pix];
    const float w = 1.f / (var_bkg + fmaxf(dv, 0.f) * inv_t);
    v[0] = w * dv * mv;
    v[1] = w * mv * mv;
    v[2] = w * dv * dv;
  }
  block_reduce_store<3>(v, partial + ((size_t)p * nblk + blockIdx.x) * 3);
}

// amp = A/B.
__global__ void solve_amp_kernel(const float* __restrict__ sums, float* __restrict__ amp, int n_points) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_points) return;
  const float A = sums[3 * p], B = sums[3 * p + 1];
  amp[p] = B > 0.f ? A / B : 0.f;
}

// sum w (d - amp m1)^2, evaluated directly: near the best fit C - A^2/B cancels in FP32.
__global__ void __launch_bounds__(kGradThreads) residual_chi2_kernel(const float* __restrict__ m1,
                                                                     const float* __restrict__ d, int npix,
                                                                     float var_bkg, float inv_t,
                                                                     const float* __restrict__ amp,
                                                                     float* __restrict__ partial, int nblk) {
  const int p = blockIdx.y;
  const int pix = blockIdx.x * blockDim.x + threadIdx.x;
  float v[1] = {0.f};
  if (pix < npix) {
    const float dv = d[pix];
    const float r = dv - amp[p] * m1[(size_t)p * npix + pix];
    v[0] = r * r / (var_bkg + fmaxf(dv, 0.f) * inv_t);
  }
  block_reduce_store<1>(v, partial + (size_t)p * nblk + blockIdx.x);
}

}  // namespace ls

using namespace ls;

namespace ls {
// The fixed subhalo field of a likelihood call: cached per handle for registered tables (their
// contents never change), recomputed into `scratch` otherwise.
static int subhalo_field(lens_sim* s, const lens_system& y, const DevSystem& d, long long n_samples,
                         float2* scratch, cudaStream_t st, float2** out) {
  if (y.subhalo_table < 0) {
    cudaError_t e = launch_subhalo_field(d, scratch, st);
    if (e != cudaSuccess) return cuda_fail(s, e, "subhalo field");
    *out = scratch;
    return LENS_OK;
  }
  lens_sim::FieldKey key;
  key.table = y.subhalo_table;
  key.nx = y.grid.nx;
  key.ny = y.grid.ny;
  key.s = y.grid.supersample;
  key.dpix = y.grid.pixel_scale;
  key.x0 = y.grid.x0;
  key.y0 = y.grid.y0;
  void* before = s->sub_field.p;
  int rc = ensure(s, s->sub_field, sizeof(float2) * (size_t)n_samples);
  if (rc) return rc;
  if (s->sub_field.p != before) s->field_key = lens_sim::FieldKey{};  // reallocated: contents gone
  *out = (float2*)s->sub_field.p;
  if (s->field_key == key) return LENS_OK;
  cudaError_t e = launch_subhalo_field(d, *out, st);
  if (e != cudaSuccess) return cuda_fail(s, e, "subhalo field");
  s->field_key = key;
  return LENS_OK;
}
}  // namespace ls

namespace ls {
// PSF step of the likelihood path on np images: the convolution (adjoint = 0) or its adjoint,
// the correlation (adjoint = 1, a convolution with the kernel turned by 180 degrees); the TMA
// kernel where it applies, else the generic one.
static cudaError_t psf_step(lens_sim* s, const float* in, float* out, int np, int ny, int nx, const PsfEntry* psf,
                            int adjoint, cudaStream_t st) {
  if (s->wait_flag_d && conv_tma_supported(in, out, ny, nx, psf->k))
    return launch_conv_tma(in, out, np, ny, nx, adjoint ? psf->dflip : psf->d, psf->k, s->wait_flag_d, s->sm_count,
                           st);
  return launch_conv(in, out, np, ny, nx, psf->d, psf->k, adjoint ? 0 : 1, st);
}
}  // namespace ls

extern "C" int lens_sim_grad(lens_sim* s, const lens_system* sys, const float* data, float sigma_bkg, float t_exp,
                             const float* params, int n_points, float* out_logL, float* out_grad, void* stream) {
  if (!s) return LENS_ERR_INVALID_ARG;
  if (!sys || !data || !params || !out_logL) return fail(s, LENS_ERR_INVALID_ARG, "NULL argument");
  if (n_points < 0 || n_points > s->max_batch)
    return fail(s, LENS_ERR_INVALID_ARG, "n_points %d not in [0, %d]", n_points, s->max_batch);
  if (!(sigma_bkg > 0.f) || !(t_exp > 0.f)) return fail(s, LENS_ERR_INVALID_ARG, "sigma_bkg and t_exp must be > 0");
  if (n_points == 0) return LENS_OK;
  DeviceGuard guard(s->device);
  if (int rw = ensure_wait_flag(s)) return rw;
  lens_system y = *sys;
  y.n_deflectors = 0;   // the free parameters replace the deflector list and source
  y.source.type = LIGHT_SERSIC;
  y.source.p[1] = 1.f;
  y.source.p[2] = 1.f;
  int rc = validate_system(s, y, true);
  if (rc) return rc;
  if (!is_device_ptr(data) || !is_device_ptr(params) || !is_device_ptr(out_logL) ||
      (out_grad && !is_device_ptr(out_grad)))
    return fail(s, LENS_ERR_INVALID_ARG, "data, params and outputs must be device memory");
  cudaStream_t st = (cudaStream_t)stream;
  const int nx = y.grid.nx, ny = y.grid.ny, ss = y.grid.supersample;
  const int npix = nx * ny;
  const long long n_samples = (long long)npix * ss * ss;
  const int nblk_l = (npix + kGradThreads - 1) / kGradThreads;
  const int nblk_b = blocks_per_point(n_samples);
  // workspace: alpha_sub | m0 | m | g_m | g_m0 | partials (per point chunk)
  const size_t sub_bytes = ((size_t)n_samples * sizeof(float2) + 255) & ~(size_t)255;
  const size_t per_point = 4 * (size_t)npix * sizeof(float) +
                           ((size_t)nblk_l + (size_t)nblk_b * LENS_N_FREE_PARAMS) * sizeof(float);
  int chunk = n_points;
  const size_t cap_target = (size_t)1 << 30;
  while (chunk > 1 && sub_bytes + per_point * chunk > cap_target) chunk = (chunk + 1) / 2;
  const size_t n_sub_max = (size_t)sub_count(s, y);
  size_t need = sub_bytes + per_point * chunk + 256 * 8;
  if ((rc = ensure(s, s->grad_ws, need))) return rc;
  if (y.subhalo_table < 0 && y.n_subhalos > 0) {
    if ((rc = ensure(s, s->tab, kTableStride * sizeof(float4) * n_sub_max))) return rc;
    if ((rc = ensure(s, s->raw_sub, 5 * sizeof(float) * n_sub_max))) return rc;
  }
  DevSystem d;
  fill_dev_system(y, d);
  d.n_defl = 0;
  if ((rc = prepare_subhalos(s, y, (float4*)s->tab.p, (float*)s->raw_sub.p, &d.sub, &d.n_sub, st))) return rc;
  char* base = (char*)s->grad_ws.p;
  float2* asub = nullptr;
  if ((rc = subhalo_field(s, y, d, n_samples, (float2*)base, st, &asub))) return rc;
  base += sub_bytes;
  float* m0 = (float*)base;
  float* m = m0 + (size_t)chunk * npix;
  float* gm = m + (size_t)chunk * npix;
  float* gm0 = gm + (size_t)chunk * npix;
  float* pl = gm0 + (size_t)chunk * npix;
  float* pg = pl + (size_t)chunk * nblk_l;
  cudaError_t e;
  PsfEntry psf_copy;
  const PsfEntry* psf = (y.psf_id >= 0 && s->res->psf(y.psf_id, &psf_copy)) ? &psf_copy : nullptr;
  for (int p0 = 0; p0 < n_points; p0 += chunk) {
    const int np = std::min(chunk, n_points - p0);
    const float* P = params + (size_t)p0 * LENS_N_FREE_PARAMS;
    forward_model_kernel<<<dim3(blocks_per_point(npix), np), kGradThreads, 0, st>>>(d, P, asub, m0, 0);
    if (psf) e = psf_step(s, m0, m, np, ny, nx, psf, 0, st);
    else e = cudaMemcpyAsync(m, m0, sizeof(float) * (size_t)np * npix, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(s, e, "model convolution");
    likelihood_kernel<<<dim3(nblk_l, np), kGradThreads, 0, st>>>(m, data, npix, sigma_bkg * sigma_bkg, 1.f / t_exp,
                                                                  out_grad ? gm : nullptr, pl, nblk_l);
    reduce_partials_kernel<<<(np + 127) / 128, 128, 0, st>>>(pl, nblk_l, 1, -0.5f, out_logL + p0, np);
    if (out_grad) {
      if (psf) e = psf_step(s, gm, gm0, np, ny, nx, psf, 1, st);
      else e = cudaMemcpyAsync(gm0, gm, sizeof(float) * (size_t)np * npix, cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return cuda_fail(s, e, "adjoint convolution");
      backward_kernel<<<dim3(nblk_b, np), kGradThreads, 0, st>>>(d, P, asub, gm0, pg, nblk_b);
      reduce_partials_kernel<<<(np * LENS_N_FREE_PARAMS + 127) / 128, 128, 0, st>>>(
          pg, nblk_b, LENS_N_FREE_PARAMS, 1.f, out_grad + (size_t)p0 * LENS_N_FREE_PARAMS, np);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(s, e, "likelihood kernels");
  }
  return LENS_OK;
}

extern "C" int lens_sim_linear_amp(lens_sim* s, const lens_system* sys, const float* data, float sigma_bkg,
                                   float t_exp, const float* params, int n_points, float* out_amp, float* out_logL,
                                   void* stream) {
  if (!s) return LENS_ERR_INVALID_ARG;
  if (!sys || !data || !params || !out_amp) return fail(s, LENS_ERR_INVALID_ARG, "NULL argument");
  if (n_points < 0 || n_points > s->max_batch)
    return fail(s, LENS_ERR_INVALID_ARG, "n_points %d not in [0, %d]", n_points, s->max_batch);
  if (!(sigma_bkg > 0.f) || !(t_exp > 0.f)) return fail(s, LENS_ERR_INVALID_ARG, "sigma_bkg and t_exp must be > 0");
  if (n_points == 0) return LENS_OK;
  DeviceGuard guard(s->device);
  if (int rw = ensure_wait_flag(s)) return rw;
  lens_system y = *sys;
  y.n_deflectors = 0;
  y.source.type = LIGHT_SERSIC;
  y.source.p[1] = 1.f;
  y.source.p[2] = 1.f;
  int rc = validate_system(s, y, true);
  if (rc) return rc;
  if (!is_device_ptr(data) || !is_device_ptr(params) || !is_device_ptr(out_amp) ||
      (out_logL && !is_device_ptr(out_logL)))
    return fail(s, LENS_ERR_INVALID_ARG, "data, params and outputs must be device memory");
  cudaStream_t st = (cudaStream_t)stream;
  const int nx = y.grid.nx, ny = y.grid.ny, ss = y.grid.supersample;
  const int npix = nx * ny;
  const long long n_samples = (long long)npix * ss * ss;
  const int nblk = (npix + kGradThreads - 1) / kGradThreads;
  const size_t sub_bytes = ((size_t)n_samples * sizeof(float2) + 255) & ~(size_t)255;
  const size_t per_point = 2 * (size_t)npix * sizeof(float) + ((size_t)nblk * 3 + 3) * sizeof(float);
  int chunk = n_points;
  while (chunk > 1 && sub_bytes + per_point * chunk > ((size_t)1 << 30)) chunk = (chunk + 1) / 2;
  if ((rc = ensure(s, s->grad_ws, sub_bytes + per_point * chunk + 256 * 4))) return rc;
  const size_t n_sub_max = (size_t)sub_count(s, y);
  if (y.subhalo_table < 0 && y.n_subhalos > 0) {
    if ((rc = ensure(s, s->tab, kTableStride * sizeof(float4) * n_sub_max))) return rc;
    if ((rc = ensure(s, s->raw_sub, 5 * sizeof(float) * n_sub_max))) return rc;
  }
  DevSystem d;
  fill_dev_system(y, d);
  d.n_defl = 0;
  if ((rc = prepare_subhalos(s, y, (float4*)s->tab.p, (float*)s->raw_sub.p, &d.sub, &d.n_sub, st))) return rc;
  char* base = (char*)s->grad_ws.p;
  float2* asub = nullptr;
  if ((rc = subhalo_field(s, y, d, n_samples, (float2*)base, st, &asub))) return rc;
  base += sub_bytes;
  float* m0 = (float*)base;
  float* m1 = m0 + (size_t)chunk * npix;
  float* part = m1 + (size_t)chunk * npix;
  float* sums = part + (size_t)chunk * nblk * 3;
  cudaError_t e;
  PsfEntry psf_copy;
  const PsfEntry* psf = (y.psf_id >= 0 && s->res->psf(y.psf_id, &psf_copy)) ? &psf_copy : nullptr;
  for (int p0 = 0; p0 < n_points; p0 += chunk) {
    const int np = std::min(chunk, n_points - p0);
    const float* P = params + (size_t)p0 * LENS_N_FREE_PARAMS;
    forward_model_kernel<<<dim3(blocks_per_point(npix), np), kGradThreads, 0, st>>>(d, P, asub, m0, 1);
    if (psf) e = psf_step(s, m0, m1, np, ny, nx, psf, 0, st);
    else e = cudaMemcpyAsync(m1, m0, sizeof(float) * (size_t)np * npix, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(s, e, "model convolution");
    normal_eq_kernel<<<dim3(nblk, np), kGradThreads, 0, st>>>(m1, data, npix, sigma_bkg * sigma_bkg, 1.f / t_exp,
                                                               part, nblk);
    reduce_partials_kernel<<<(np * 3 + 127) / 128, 128, 0, st>>>(part, nblk, 3, 1.f, sums, np);
    solve_amp_kernel<<<(np + 127) / 128, 128, 0, st>>>(sums, out_amp + p0, np);
    if (out_logL) {
      residual_chi2_kernel<<<dim3(nblk, np), kGradThreads, 0, st>>>(m1, data, npix, sigma_bkg * sigma_bkg,
                                                                      1.f / t_exp, out_amp + p0, part, nblk);
      reduce_partials_kernel<<<(np + 127) / 128, 128, 0, st>>>(part, nblk, 1, -0.5f, out_logL + p0, np);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(s, e, "linear amplitude kernels");
  }
  return LENS_OK;
}

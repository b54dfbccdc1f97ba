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
// The per-sample local Jacobians dalpha_EPL/dp and dI/d(p_src, beta) come from a forward-mode
// dual type; every reduction is a fixed-order two-stage tree (deterministic).
#include <algorithm>

#include "dual.cuh"
#include "kernels.h"
#include "lens_sim.h"
#include "sim_internal.h"

namespace ls {

constexpr int kGradThreads = 256;
using D6 = Dn<6>;

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

// Fixed subhalo deflection at every sample (sample order: row, column, sub-row, sub-column).
__global__ void __launch_bounds__(256) subhalo_field_kernel(const __grid_constant__ DevSystem sys,
                                                            float2* __restrict__ out, long long n_samples) {
  __shared__ float4 s_sub[8][32][kSubStride];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long first = (long long)blockIdx.x * blockDim.x + w * 32;
  if (first >= n_samples) return;
  const long long idx = first + lane;
  float px = 0.f, py = 0.f;
  int pix;
  if (idx < n_samples) sample_coords(sys, idx, px, py, pix);
  float ax = 0.f, ay = 0.f;
  const float4* __restrict__ mid_tab = sys.sub + (size_t)kSubStride * sys.n_sub;
  for (int base = 0; base < sys.n_sub; base += 32) {
    const int t = base + lane;
    if (t < sys.n_sub) {
#pragma unroll
      for (int c = 0; c < kSubStride; ++c) s_sub[w][lane][c] = __ldg(sys.sub + (size_t)kSubStride * t + c);
    }
    __syncwarp();
    const int cnt = min(32, sys.n_sub - base);
    for (int q = 0; q < cnt; ++q)
      tnfw_pair(px, py, s_sub[w][q], mid_tab + (size_t)kMidStride * (base + q), ax, ay);
    __syncwarp();
  }
  if (idx < n_samples) out[idx] = make_float2(ax, ay);
}

// ---------------------------------------------------------------------------- forward model
__device__ __forceinline__ float model_sample(float x, float y, float2 asub, const float* __restrict__ P) {
  float ex, ey;
  {
    float q, phi;
    e1e2_to_qphi(P[2], P[3], q, phi);
    alpha_epl(x, y, P[0], P[1], q, phi, P[4], P[5], ex, ey);
  }
  const float bx = x - ex - (P[6] * x + P[7] * y) - asub.x;
  const float by = y - ey - (P[7] * x - P[6] * y) - asub.y;
  float q, phi;
  e1e2_to_qphi(P[11], P[12], q, phi);
  return sersic(bx, by, P[8], P[9], P[10], q, phi, P[13], P[14]);
}

__global__ void __launch_bounds__(kGradThreads) forward_model_kernel(const __grid_constant__ DevSystem g,
                                                                     const float* __restrict__ params,
                                                                     const float2* __restrict__ asub,
                                                                     float* __restrict__ m0, int unit_amp) {
  __shared__ float P[LENS_N_FREE_PARAMS];
  const int p = blockIdx.y;
  if (threadIdx.x < LENS_N_FREE_PARAMS) P[threadIdx.x] = params[p * LENS_N_FREE_PARAMS + threadIdx.x];
  if (unit_amp && threadIdx.x == 8) P[8] = 1.f;  // linear solve: the model per unit source amplitude
  __syncthreads();
  const int npix = g.nx * g.ny;
  const int pix = blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= npix) return;
  const int s2 = g.s * g.s;
  float acc = 0.f;
  for (int k = 0; k < s2; ++k) {
    const long long idx = (long long)pix * s2 + k;
    float x, y;
    int pp;
    sample_coords(g, idx, x, y, pp);
    acc += model_sample(x, y, asub[idx], P);
  }
  m0[(size_t)p * npix + pix] = acc * (g.dpix * g.dpix / (float)s2);
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
__device__ __forceinline__ void e1e2_to_qphi_d(const D6& e1, const D6& e2, D6& q, D6& phi) {
  phi = datan2(e2, e1) * 0.5f;
  const D6 c = dsqrt(e1 * e1 + e2 * e2);
  q = (1.f - c) / (1.f + c);
}

// EPL deflection with tangents along (theta_E, gamma, e1, e2, cx, cy) at a fixed point.
__device__ __noinline__ void epl_alpha_jac(float x, float y, const float* __restrict__ P, D6& ax, D6& ay) {
  const D6 thetaE = dvar<6>(P[0], 0), gamma = dvar<6>(P[1], 1);
  const D6 e1 = dvar<6>(P[2], 2), e2 = dvar<6>(P[3], 3);
  const D6 cx = dvar<6>(P[4], 4), cy = dvar<6>(P[5], 5);
  D6 q, phi;
  e1e2_to_qphi_d(e1, e2, q, phi);
  const D6 cp = dcos(phi), sp = dsin(phi);
  const D6 dx = x - cx, dy = y - cy;
  const D6 xp = cp * dx + sp * dy, yp = sp * (-1.f) * dx + cp * dy;
  const D6 R = dsqrt(q * q * xp * xp + yp * yp);
  if (R.v < 1e-12f) { ax = dconst<6>(0.f); ay = dconst<6>(0.f); return; }
  const D6 t = gamma - 1.f;
  const D6 b = thetaE * dsqrt(q);
  const D6 iR = inv(R);
  const D6 er = q * xp * iR, ei = yp * iR;
  const D6 f = (1.f - q) / (1.f + q);
  const D6 zr = -f * (er * er - ei * ei), zi = -f * (2.f * er * ei);
  D6 omr = er, omi = ei, sr = er, si = ei;
  const int nt = epl_terms(f.v) + 4;  // tangents converge like n f^(n-1)
  for (int n = 1; n <= nt; ++n) {
    const D6 coef = ((2.f * n - 2.f) + t) / ((2.f * n + 2.f) - t);
    const D6 nr = coef * (omr * zr - omi * zi);
    const D6 ni = coef * (omr * zi + omi * zr);
    omr = nr;
    omi = ni;
    sr = sr + omr;
    si = si + omi;
  }
  const D6 pref = (2.f * b / (1.f + q)) * dexp((t - 1.f) * dlog(b * iR));
  const D6 apx = pref * sr, apy = pref * si;
  ax = cp * apx - sp * apy;
  ay = sp * apx + cp * apy;
}

// Sersic with tangents along (R_s, n, e1, e2, beta_x, beta_y); dI/damp = I/amp and
// dI/dc = -dI/dbeta follow without tangents.
__device__ __noinline__ D6 sersic_jac(float bx, float by, const float* __restrict__ P) {
  const D6 Rs = dvar<6>(P[9], 0), n = dvar<6>(P[10], 1);
  const D6 e1 = dvar<6>(P[11], 2), e2 = dvar<6>(P[12], 3);
  const D6 Bx = dvar<6>(bx, 4), By = dvar<6>(by, 5);
  D6 q, phi;
  e1e2_to_qphi_d(e1, e2, q, phi);
  const D6 cp = dcos(phi), sp = dsin(phi);
  const D6 dx = Bx - P[13], dy = By - P[14];
  const D6 xp = cp * dx + sp * dy, yp = sp * (-1.f) * dx + cp * dy;
  const D6 R = dsqrt(q * xp * xp + yp * yp / q);
  const D6 bn = 1.9992f * n - 0.3271f;
  if (R.v <= 0.f) return dexp(bn) * P[8];
  const D6 pw = dexp(dlog(R / Rs) / n);
  return dexp(-bn * (pw - 1.f)) * P[8];
}

__global__ void __launch_bounds__(kGradThreads) backward_kernel(const __grid_constant__ DevSystem g,
                                                                const float* __restrict__ params,
                                                                const float2* __restrict__ asub,
                                                                const float* __restrict__ gm0,
                                                                float* __restrict__ partial, int nblk) {
  __shared__ float P[LENS_N_FREE_PARAMS];
  const int p = blockIdx.y;
  if (threadIdx.x < LENS_N_FREE_PARAMS) P[threadIdx.x] = params[p * LENS_N_FREE_PARAMS + threadIdx.x];
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
    D6 ax, ay;
    epl_alpha_jac(x, y, P, ax, ay);
    const float2 as = asub[idx];
    const float bx = x - ax.v - (P[6] * x + P[7] * y) - as.x;
    const float by = y - ay.v - (P[7] * x - P[6] * y) - as.y;
    const D6 I = sersic_jac(bx, by, P);
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
    subhalo_field_kernel<<<(unsigned)((n_samples + 255) / 256), 256, 0, st>>>(d, scratch, n_samples);
    cudaError_t e = cudaGetLastError();
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
  subhalo_field_kernel<<<(unsigned)((n_samples + 255) / 256), 256, 0, st>>>(d, *out, n_samples);
  cudaError_t e = cudaGetLastError();
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
  const int nblk_b = (int)std::min<long long>((n_samples + kGradThreads - 1) / kGradThreads, 64);
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
    forward_model_kernel<<<dim3((npix + kGradThreads - 1) / kGradThreads, np), kGradThreads, 0, st>>>(d, P, asub, m0, 0);
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
    forward_model_kernel<<<dim3(nblk, np), kGradThreads, 0, st>>>(d, P, asub, m0, 1);
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
